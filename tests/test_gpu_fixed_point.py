"""BlockBP at its fixed point on the Kagome workloads, GPU against the FP64
oracle's stored values (tests/golden, written by make_kagome_golden.py from
oracle/ alone).

Kagome 6 x 2 super-cell, parallelogram blocks of L = 2 (3 blocks of 12
sites), d = 2, dimer-singlet tensors with 1e-2 noise:

* D = 4, chi = 32, FP64 path, iterated to tol 1e-10 (Alg. 1 with the
  convergence criterion of the BP update): the iteration count within one of
  the oracle's, and every <S^z_i>, every bond <S_i . S_j>, the energy per
  site and the Bethe log-norm within 1e-10.
* the same in the mixed-precision modes (TF32 and BF16 contractions),
  iterated until the largest message change is below 1e-5 (their messages
  are complex64, whose rounding sets a floor near 1e-6): every <S^z_i>, every
  bond energy and the energy per site within 1e-5 of the FP64 fixed point.
* D = 6, chi = 64, mixed precision, two iterations from the initial messages:
  every <S^z_i> and a fixed sample of bonds within 1e-5 of the oracle.
"""
import json
import os

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")

HERE = os.path.dirname(os.path.abspath(__file__))
SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def kagome_ctx(D, chi, precision):
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(len(nb), D, seed=7)
    ctx = P.bbp_create_peps(P.KAGOME, 6, 2, 1, 2, D, t)
    P.bbp_partition_blocks(ctx, 2, 2)
    P.bbp_set_options(ctx, chi, precision)
    P.bbp_init_messages(ctx, em)
    return ctx


def observables(ctx, g, bonds):
    sz = np.array([P.bbp_expect_local(ctx, SZ, [i]).real for i in range(36)])
    # three product insertions S^a (x) S^a per bond, the scheme of the
    # oracle's bond energy (a truncated sweep is not linear in the inserted
    # operator)
    be = P.bbp_bond_energies(ctx, [(b[0], b[1]) for b in bonds])
    return sz, be


def test_config2_fp64_fixed_point():
    g = golden("kagome_D4_chi32_fixed_point.json")
    ctx = kagome_ctx(4, 32, P.FP64)
    try:
        it, err, conv = P.bbp_iterate(ctx, 1e-10, 30)
        print(f"FP64 D=4 chi=32: {it} iterations (oracle {g['iterations']}), error {err:.3e}")
        assert conv and err <= 1e-10
        assert abs(it - g["iterations"]) <= 1
        sz, be = observables(ctx, g, g["bonds"])
        dsz = np.abs(sz - np.array([v[0] for v in g["sz"]])).max()
        dbe = np.abs(be - np.array([v[0] for v in g["bond_energy"]])).max()
        de = abs(P.bbp_energy_per_site(ctx) - g["energy_per_site"])
        dn = abs(P.bbp_norm(ctx) - g["log_norm"])
        print(f"  max|d<Sz>| {dsz:.2e}  max|d<S.S>| {dbe:.2e}  |dE/site| {de:.2e}  |d log Z| {dn:.2e}")
        assert dsz < 1e-10 and dbe < 1e-10 and de < 1e-10 and dn < 1e-10
    finally:
        P.bbp_destroy(ctx)


@pytest.mark.parametrize("mode", ["TF32", "BF16"])
def test_config2_mixed_fixed_point(mode):
    g = golden("kagome_D4_chi32_fixed_point.json")
    ctx = kagome_ctx(4, 32, getattr(P, mode))
    try:
        it, err, conv = P.bbp_iterate(ctx, 1e-5, 30)
        print(f"{mode} D=4 chi=32: {it} iterations to error {err:.3e}")
        assert conv
        sz, be = observables(ctx, g, g["bonds"])
        dsz = np.abs(sz - np.array([v[0] for v in g["sz"]])).max()
        dbe = np.abs(be - np.array([v[0] for v in g["bond_energy"]])).max()
        de = abs(P.bbp_energy_per_site(ctx) - g["energy_per_site"])
        print(f"  vs FP64 fixed point: max|d<Sz>| {dsz:.2e}  max|d<S.S>| {dbe:.2e}  |dE/site| {de:.2e}")
        assert dsz < 1e-5 and dbe < 1e-5 and de < 1e-5
    finally:
        P.bbp_destroy(ctx)


@pytest.mark.parametrize("mode", ["TF32", "BF16"])
def test_config3_mixed_two_iterations(mode):
    """Kagome D = 6, chi = 64 (splits of 2304 x 2304): the randomised,
    tensor-core path against the FP64 oracle on every site and the sampled
    bonds, after the same two iterations."""
    g = golden("kagome_D6_chi64_2it.json")
    ctx = kagome_ctx(6, 64, getattr(P, mode))
    try:
        it, err, _ = P.bbp_iterate(ctx, 0.0, 2)
        assert it == 2
        print(f"{mode} D=6 chi=64: error after 2 iterations {err:.6e} (oracle {g['errors'][-1]:.6e})")
        sz, be = observables(ctx, g, g["bonds"])
        dsz = np.abs(sz - np.array([v[0] for v in g["sz"]])).max()
        dbe = np.abs(be - np.array([v[0] for v in g["bond_energy"]])).max()
        print(f"  max|d<Sz>| {dsz:.2e} over 36 sites, max|d<S.S>| {dbe:.2e} over {len(be)} bonds")
        assert dsz < 1e-5 and dbe < 1e-5
        assert abs(err - g["errors"][-1]) < 1e-4 * max(1.0, g["errors"][-1])
    finally:
        P.bbp_destroy(ctx)
