"""The mixed-precision paths (BBP_FP32, BBP_TF32, BBP_BF16) against the FP64
oracle.

Same seeded inputs, same number of synchronous iterations; the bound of the
mixed-precision path is 1e-5 on every reported energy and <S^z>.  Messages
are compared too (dense, gauge-invariant) and the largest difference is
printed: it is a measurement, the 1e-5 bound applies to observables.
TF32 / BF16 run the absorb contraction on the tensor cores (split operands).
"""
import functools
import numpy as np
import pytest

import synthetic as syn
from oracle import tn
from oracle.blockbp import BlockBP
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")

BOUND = 1e-5
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def run(kind, args, t, em, chi, iters, precision):
    d, D = t.shape[1], t.shape[2]
    if kind == "square":
        ctx = P.bbp_create_peps(P.SQUARE, args[0], args[1], 0, d, D, t)
        P.bbp_partition_blocks(ctx, args[2], args[3])
    else:
        ctx = P.bbp_create_peps(P.KAGOME, args[0], args[1], 1, d, D, t)
        P.bbp_partition_blocks(ctx, args[2], args[2])
    P.bbp_set_options(ctx, chi, precision)
    P.bbp_init_messages(ctx, em)
    P.bbp_iterate(ctx, 0.0, iters)
    return ctx


def msg_diff(ctx, bb):
    worst = 0.0
    for (bid, face), m in bb.msgs.items():
        g = P.bbp_get_message(ctx, bid, face)
        worst = max(worst, float(np.linalg.norm(tn.mps_dense(g) - tn.mps_dense(m))))
    return worst


MODES = ("FP32", "TF32", "BF16")


@functools.lru_cache(maxsize=None)
def oracle_square():
    t = syn.gaussian_peps(36, 2, 2, seed=1)
    em = syn.initial_edge_matrices(36, 2, seed=11)
    bb = BlockBP(Geometry.square(6, 6, 3, 3), t, chi=8)
    bb.init_messages(em)
    for _ in range(12):
        bb.step()
    return t, em, bb, [bb.sz(g) for g in range(36)], bb.energy_per_site().real


@functools.lru_cache(maxsize=None)
def oracle_kagome(D, chi, iters):
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(36, D, seed=7)
    bb = BlockBP(Geometry.kagome(6, 2, 2), t, chi=chi)
    bb.init_messages(em)
    for _ in range(iters):
        bb.step()
    sites = (0, 7, 13, 22, 35)
    return t, em, bb, {g: bb.sz(g) for g in sites}, bb.energy_per_site().real


@pytest.mark.parametrize("mode", list(MODES))
def test_mixed_square_config1(mode):
    t, em, bb, sz_ref, e_ref = oracle_square()
    ctx = run("square", (6, 6, 3, 3), t, em, 8, 12, getattr(P, mode))
    try:
        print(f"config 1 {mode} message diff", msg_diff(ctx, bb))
        errs = [abs(P.bbp_expect_local(ctx, SZ, [g]) - sz_ref[g]) for g in range(36)]
        de = abs(P.bbp_energy_per_site(ctx) - e_ref)
        print(f"config 1 {mode}: max |d<Sz>| = {max(errs):.2e}  |dE/site| = {de:.2e}")
        assert max(errs) < BOUND and de < BOUND
    finally:
        P.bbp_destroy(ctx)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("D,chi,iters", [(2, 8, 6), (4, 32, 3)])
def test_mixed_kagome(D, chi, iters, mode):
    """Kagome dimer-singlet + 1e-2 noise; D = 4, chi = 32 uses the randomised
    truncation on the 512 x 512 bulk matrices."""
    t, em, bb, sz_ref, e_ref = oracle_kagome(D, chi, iters)
    ctx = run("kagome", (6, 2, 2), t, em, chi, iters, getattr(P, mode))
    try:
        print(f"Kagome D={D} chi={chi} {mode} message diff", msg_diff(ctx, bb))
        e_gpu = P.bbp_energy_per_site(ctx)
        dsz = max(abs(P.bbp_expect_local(ctx, SZ, [g]) - v) for g, v in sz_ref.items())
        print(f"Kagome D={D} chi={chi} {mode}: E/site {e_gpu:.10f} vs {e_ref:.10f} "
              f"(|dE| {abs(e_gpu - e_ref):.2e}); max |d<Sz>| {dsz:.2e}")
        assert abs(e_gpu - e_ref) < BOUND
        assert dsz < BOUND
    finally:
        P.bbp_destroy(ctx)


def test_graph_replay_matches_eager():
    """The captured-graph iteration computes what eager launches compute."""
    t, em, _, _, _ = oracle_square()
    out = []
    for graphs in (True, False):
        ctx = P.bbp_create_peps(P.SQUARE, 6, 6, 0, 2, 2, t)
        P.bbp_partition_blocks(ctx, 3, 3)
        P.bbp_set_options(ctx, 8, P.FP64)
        P.bbp_set_execution(ctx, graphs, 16)
        P.bbp_init_messages(ctx, em)
        P.bbp_iterate(ctx, 0.0, 6)
        out.append({(b, f): tn.mps_dense(P.bbp_get_message(ctx, b, f)) for (b, f) in oracle_square()[2].msgs})
        P.bbp_destroy(ctx)
    worst = max(float(np.linalg.norm(out[0][k] - out[1][k])) for k in out[0])
    print("graph vs eager message diff", worst)
    assert worst < 1e-12
