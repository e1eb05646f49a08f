"""End-to-end parity of the FP64 GPU BlockBP path with the FP64 oracle.

Both sides receive the same seeded PEPS tensors and initial edge matrices and
run the same number of synchronous iterations; messages (unit norm, phase
fixed, compared as dense vectors over their fused legs), local observables
and the Bethe log-norm must agree to 1e-10 (the FP64 tolerance of the
method's GPU path).  Messages are gauge-invariant objects, so the comparison
is independent of the (different) SVD/QR phase conventions of both sides.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import exact, tn
from oracle.blockbp import BlockBP
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")

TOL = 1e-10
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def gpu_run(kind, geom_args, t, em, chi, iters, tol=0.0):
    d, D = t.shape[1], t.shape[2]
    if kind == "square":
        Lx, Ly, bx, by = geom_args[:4]
        per = geom_args[4] if len(geom_args) > 4 else 0
        ctx = P.bbp_create_peps(P.SQUARE, Lx, Ly, per, d, D, t)
        P.bbp_partition_blocks(ctx, bx, by)
    else:
        Lx, Ly, L = geom_args
        ctx = P.bbp_create_peps(P.KAGOME, Lx, Ly, 1, d, D, t)
        P.bbp_partition_blocks(ctx, L, L)
    P.bbp_set_options(ctx, chi)
    P.bbp_init_messages(ctx, em)
    it, err, conv = P.bbp_iterate(ctx, tol, iters)
    return ctx, it, err


def compare_messages(ctx, bb, tol=TOL):
    worst = 0.0
    for (bid, face), m in bb.msgs.items():
        g = P.bbp_get_message(ctx, bid, face)
        vg, vo = tn.mps_dense(g), tn.mps_dense(m)
        worst = max(worst, float(np.linalg.norm(vg - vo)))
    assert worst <= tol, f"largest message difference {worst:.3e}"
    return worst


def test_config1_square_6x6_fp64():
    """6 x 6 open square PEPS, d = 2, D = 2, Gaussian tensors / sigma_max,
    2 x 2 blocks of 3 x 3 sites, chi = 8, FP64: messages, all <S^z>, the
    energy per site and the log-norm equal the oracle to 1e-10."""
    n = 36
    t = syn.gaussian_peps(n, 2, 2, seed=1)
    em = syn.initial_edge_matrices(n, 2, seed=11)
    geom = Geometry.square(6, 6, 3, 3)
    bb = BlockBP(geom, t, chi=8)
    bb.init_messages(em)
    errs = [bb.step() for _ in range(12)]
    ctx, it, err = gpu_run("square", (6, 6, 3, 3), t, em, chi=8, iters=12)
    try:
        assert it == 12
        assert abs(err - errs[-1]) < 1e-9
        compare_messages(ctx, bb)
        for g in range(n):
            got = P.bbp_expect_local(ctx, SZ, [g])
            assert abs(got - bb.sz(g)) < TOL
        e_gpu = P.bbp_energy_per_site(ctx)
        assert abs(e_gpu - bb.energy_per_site().real) < TOL
        assert abs(P.bbp_norm(ctx) - bb.log_norm()) < 1e-9
        # report the BlockBP error against the exact contraction (not a parity claim)
        ex = [exact.expect(geom.lattice, t, {g: SZ}).real for g in range(0, n, 7)]
        bp = [P.bbp_expect_local(ctx, SZ, [g]).real for g in range(0, n, 7)]
        print("max |<Sz>_BlockBP - <Sz>_exact| =", max(abs(a - b) for a, b in zip(ex, bp)))
    finally:
        P.bbp_destroy(ctx)


def test_square_converges_with_tolerance():
    n = 36
    t = syn.gaussian_peps(n, 2, 2, seed=1)
    em = syn.initial_edge_matrices(n, 2, seed=11)
    bb = BlockBP(Geometry.square(6, 6, 3, 3), t, chi=8)
    bb.init_messages(em)
    it_o, err_o = bb.run(1e-10, 60)
    ctx, it, err = gpu_run("square", (6, 6, 3, 3), t, em, chi=8, iters=60, tol=1e-10)
    try:
        assert err <= 1e-10 and err_o <= 1e-10
        assert abs(it - it_o) <= 1
        compare_messages(ctx, bb)
    finally:
        P.bbp_destroy(ctx)


@pytest.mark.parametrize("layout", [(3, 3, 1, 1), (4, 4, 2, 2), (6, 2, 2, 2), (4, 4, 2, 2, 1)])
def test_square_layouts(layout):
    """1 x 1 blocks (BP), ragged 2 x 2 blocks, a chain of blocks (exact), a torus."""
    Lx, Ly = layout[:2]
    per = layout[4] if len(layout) > 4 else 0
    n = Lx * Ly
    t = syn.gaussian_peps(n, 2, 2, seed=5)
    em = syn.initial_edge_matrices(n, 2, seed=6)
    bb = BlockBP(Geometry.square(Lx, Ly, layout[2], layout[3], periodic=bool(per)), t, chi=6)
    bb.init_messages(em)
    for _ in range(4):
        bb.step()
    ctx, it, err = gpu_run("square", layout, t, em, chi=6, iters=4)
    try:
        compare_messages(ctx, bb)
        for g in (0, n - 1):
            assert abs(P.bbp_expect_local(ctx, SZ, [g]) - bb.sz(g)) < TOL
    finally:
        P.bbp_destroy(ctx)


def test_product_state_d1():
    """D = 1: all bonds trivial; the GPU path handles dimension-1 legs."""
    rng = np.random.default_rng(41)
    v = rng.standard_normal((16, 2)) + 1j * rng.standard_normal((16, 2))
    t = v.reshape(16, 2, 1, 1, 1, 1)
    em = syn.initial_edge_matrices(16, 1, seed=42)
    ctx, it, err = gpu_run("square", (4, 4, 2, 2), t, em, chi=4, iters=3)
    try:
        assert err < 1e-14
        for g in range(16):
            ref = np.vdot(v[g], SZ @ v[g]) / np.vdot(v[g], v[g])
            assert abs(P.bbp_expect_local(ctx, SZ, [g]) - ref) < 1e-13
    finally:
        P.bbp_destroy(ctx)


def test_kagome_dimer_small():
    """Kagome 6 x 2 unit cells (3 parallelogram blocks of 12 sites, periodic
    super-cell), D = 2 dimer singlets + 1e-2 noise, chi = 8."""
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, 2, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(36, 2, seed=7)
    bb = BlockBP(Geometry.kagome(6, 2, 2), t, chi=8)
    bb.init_messages(em)
    for _ in range(5):
        bb.step()
    ctx, it, err = gpu_run("kagome", (6, 2, 2), t, em, chi=8, iters=5)
    try:
        compare_messages(ctx, bb)
        assert abs(P.bbp_energy_per_site(ctx) - bb.energy_per_site().real) < TOL
        for g in (0, 13, 35):
            assert abs(P.bbp_expect_local(ctx, SZ, [g]) - bb.sz(g)) < TOL
    finally:
        P.bbp_destroy(ctx)


def test_kagome_dimer_exact_energy():
    """Noise 0: BlockBP is exact on the dimer covering, energy/site -3/8."""
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, 2, seed=2, noise=0.0, noise_seed=0)
    em = syn.initial_edge_matrices(36, 2, seed=7)
    ctx, it, err = gpu_run("kagome", (6, 2, 2), t, em, chi=8, iters=6, tol=1e-12)
    try:
        assert abs(P.bbp_energy_per_site(ctx) + 0.375) < 1e-12
    finally:
        P.bbp_destroy(ctx)


def test_config2_kagome_d4_chi32_two_iterations():
    """Kagome D = 4, chi = 32 (the production shape: 512 x 512 SVDs), FP64:
    the first two iterations (bond-1 start, then full-bond inputs) match."""
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, 4, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(36, 4, seed=7)
    bb = BlockBP(Geometry.kagome(6, 2, 2), t, chi=32)
    bb.init_messages(em)
    for _ in range(2):
        bb.step()
    ctx, it, err = gpu_run("kagome", (6, 2, 2), t, em, chi=32, iters=2)
    try:
        compare_messages(ctx, bb)
    finally:
        P.bbp_destroy(ctx)


def test_single_block_sweep_exact():
    """A block covering a 3 x 3 open lattice with chi above every rank gives the
    exact <S^z> (no messages at all: every face is open)."""
    t = syn.gaussian_peps(9, 2, 2, seed=12)
    em = syn.initial_edge_matrices(9, 2, seed=13)
    geom = Geometry.square(3, 3, 3, 3)
    ctx, it, err = gpu_run("square", (3, 3, 3, 3), t, em, chi=64, iters=1)
    try:
        for g in range(9):
            ref = exact.expect(geom.lattice, t, {g: SZ})
            assert abs(P.bbp_expect_local(ctx, SZ, [g]) - ref) < 1e-11
        rho = P.bbp_block_rdm(ctx, 0, [4, 5])
        ref = exact.rdm(geom.lattice, t, [4, 5])
        assert np.abs(rho - ref / np.trace(ref)).max() < 1e-11
    finally:
        P.bbp_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_fuse_on_the_fly_matches_cached(prec):
    """With the fused-tensor cache off, every site is fused right before its
    absorb each iteration: the same numbers reach the same kernels, so the
    messages and the energy are unchanged (FP64 and TF32)."""
    n = 36
    t = syn.gaussian_peps(n, 2, 3, seed=8)
    em = syn.initial_edge_matrices(n, 3, seed=18)
    out = []
    for cache in (None, 0):
        ctx = P.bbp_create_peps(P.SQUARE, 6, 6, 0, 2, 3, t)
        P.bbp_partition_blocks(ctx, 3, 3)
        if cache is not None:
            P.bbp_set_fuse_cache(ctx, cache)
        P.bbp_set_options(ctx, 8, prec)
        P.bbp_init_messages(ctx, em)
        P.bbp_iterate(ctx, 0.0, 5)
        msgs = {}
        for b in range(4):
            for f in range(4):
                try:
                    msgs[(b, f)] = tn.mps_dense(P.bbp_get_message(ctx, b, f))
                except P.BBPError:
                    pass
        out.append((msgs, P.bbp_energy_per_site(ctx)))
        P.bbp_destroy(ctx)
    worst = max(float(np.abs(out[0][0][k] - out[1][0][k]).max()) for k in out[0][0])
    print(f"precision {prec}: on-the-fly vs cached fusion: message diff {worst:.2e}, "
          f"|dE| {abs(out[0][1] - out[1][1]):.2e}")
    assert worst <= 1e-14 and abs(out[0][1] - out[1][1]) <= 1e-14
