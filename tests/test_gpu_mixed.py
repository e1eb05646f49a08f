"""The complex64 path (BBP_FP32) against the FP64 oracle.

Same seeded inputs, same number of synchronous iterations; the bound of the
mixed-precision path is 1e-5 on every reported energy and <S^z>.  Messages
are compared too (dense, gauge-invariant) and the largest difference is
printed: it is a measurement, the 1e-5 bound applies to observables.
"""
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


def test_fp32_square_config1():
    t = syn.gaussian_peps(36, 2, 2, seed=1)
    em = syn.initial_edge_matrices(36, 2, seed=11)
    bb = BlockBP(Geometry.square(6, 6, 3, 3), t, chi=8)
    bb.init_messages(em)
    for _ in range(12):
        bb.step()
    ctx = run("square", (6, 6, 3, 3), t, em, 8, 12, P.FP32)
    try:
        print("config 1 FP32 message diff", msg_diff(ctx, bb))
        errs = [abs(P.bbp_expect_local(ctx, SZ, [g]) - bb.sz(g)) for g in range(36)]
        de = abs(P.bbp_energy_per_site(ctx) - bb.energy_per_site().real)
        print("config 1 FP32: max |d<Sz>| =", max(errs), " |dE/site| =", de)
        assert max(errs) < BOUND and de < BOUND
    finally:
        P.bbp_destroy(ctx)


@pytest.mark.parametrize("D,chi,iters", [(2, 8, 6), (4, 32, 3)])
def test_fp32_kagome(D, chi, iters):
    """Kagome dimer-singlet + 1e-2 noise; D = 4, chi = 32 uses the randomised
    truncation on the 512 x 512 bulk matrices."""
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(36, D, seed=7)
    bb = BlockBP(Geometry.kagome(6, 2, 2), t, chi=chi)
    bb.init_messages(em)
    for _ in range(iters):
        bb.step()
    ctx = run("kagome", (6, 2, 2), t, em, chi, iters, P.FP32)
    try:
        print(f"Kagome D={D} chi={chi} FP32 message diff", msg_diff(ctx, bb))
        e_gpu = P.bbp_energy_per_site(ctx)
        e_ref = bb.energy_per_site().real
        dsz = max(abs(P.bbp_expect_local(ctx, SZ, [g]) - bb.sz(g)) for g in (0, 7, 13, 22, 35))
        print(f"Kagome D={D} chi={chi} FP32: E/site {e_gpu:.10f} vs {e_ref:.10f}; max |d<Sz>| {dsz:.2e}")
        assert abs(e_gpu - e_ref) < BOUND
        assert dsz < BOUND
    finally:
        P.bbp_destroy(ctx)
