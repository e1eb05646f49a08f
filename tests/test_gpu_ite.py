"""ITE with ALS on the GPU (bbp_ite_bond, bbp_ite) against the oracle (Ch. 3, Alg. 2).

FP64 mode.  One bond update: the GPU's Phi history (start, then every ALS
half-step, a fixed number of sweeps) equals the oracle's ALS on the same
Edge TN to 1e-9 relative, and the energy after the update equals the
oracle's.  Full ITE: the energy per site after every time step equals the
oracle's full ITE on the same inputs, and reaches the ground states the
oracle's pins fix (two spins: the singlet, -3/8 per site; three: -1/3).
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import core as C
from oracle import ite
from oracle.blockbp import BlockBP
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def _pair(kind, args, D, chi, iters, seed):
    geom = Geometry.square(*args) if kind == "square" else Geometry.kagome(*args)
    n = geom.n_sites
    t = syn.gaussian_peps(n, 2, D, seed=seed)
    em = syn.initial_edge_matrices(n, D, seed=seed + 1)
    bb = BlockBP(geom, t, chi=chi)
    bb.init_messages(em)
    for _ in range(iters):
        bb.step()
    if kind == "square":
        ctx = P.bbp_create_peps(P.SQUARE, args[0], args[1], 0, 2, D, t)
        P.bbp_partition_blocks(ctx, args[2], args[3])
    else:
        ctx = P.bbp_create_peps(P.KAGOME, args[0], args[1], 1, 2, D, t)
        P.bbp_partition_blocks(ctx, args[2], args[2])
    P.bbp_set_options(ctx, chi, P.FP64)
    P.bbp_init_messages(ctx, em)
    if iters:
        P.bbp_iterate(ctx, 0.0, iters)
    return geom, bb, ctx, t


def _oracle_als(bb, g1, k1, G, sweeps):
    coords, key1, key2 = bb.bond_region(g1, k1)
    env = C.CoreEnv(bb, coords, [key1, key2])
    N, _, _ = env.edge(key1, key2)
    r1, r2 = env.sites[key1], env.sites[key2]
    joint = next(iter(set(r1.labels) & set(r2.labels)))
    s1, s2 = r1.labels.index(joint), r2.labels.index(joint)
    t1, t2 = bb.tc[r1.gid], bb.tc[r2.gid]
    dims1 = [t1.shape[1 + s] for s in range(4) if s != s1]
    dims2 = [t2.shape[1 + s] for s in range(4) if s != s2]
    a, b, hist = ite.als(t1, t2, s1, s2, N, dims1, dims2, G, bb.D, max_sweeps=sweeps, tol=0.0)
    return r1.gid, r2.gid, a, b, hist


CASES = [
    ("square", (3, 3, 3, 3), 2, 16, 0, 5, [(4, 1), (4, 0), (0, 1), (8, 3)]),
    ("square", (6, 6, 3, 3), 2, 8, 2, 1, [(7, 1), (14, 0)]),
    ("kagome", (6, 2, 2), 2, 16, 2, 7, [(6, 0), (7, 1), (8, 1)]),
]


@pytest.mark.parametrize("kind,args,D,chi,iters,seed,bonds", CASES)
def test_ite_bond_matches_oracle(kind, args, D, chi, iters, seed, bonds):
    G = ite.gate(ite.heisenberg_h(), 0.3)
    worst = 0.0
    for (g1, k1) in bonds:
        geom, bb, ctx, t = _pair(kind, args, D, chi, iters, seed)
        try:
            hist = P.bbp_ite_bond(ctx, g1, k1, G, max_sweeps=6, tol=0.0)
            ga, gb, a, b, hist_o = _oracle_als(bb, g1, k1, G, 6)
            assert len(hist) == len(hist_o)
            rel = max(abs(x - y) for x, y in zip(hist, hist_o)) / abs(hist_o[0])
            assert rel < 1e-9, rel
            worst = max(worst, rel)
            if kind == "square" and args[:2] == (3, 3):     # one open block: the energy is exact
                t2 = np.array(t)
                ite._put(t2, ga, a)
                ite._put(t2, gb, b)
                bb2 = BlockBP(geom, t2, chi=chi)
                e_or = bb2.energy_per_site().real
                e_gpu = P.bbp_energy_per_site(ctx)
                assert abs(e_gpu - e_or) < 1e-9, (e_gpu, e_or)
        finally:
            P.bbp_destroy(ctx)
    print(f"ITE bond {kind} {args}: largest relative Phi difference {worst:.2e}")


def _full(geom_args, dts, seed=3):
    geom = Geometry.square(*geom_args)
    n = geom.n_sites
    t = syn.gaussian_peps(n, 2, 2, seed=seed)
    em = syn.initial_edge_matrices(n, 2, seed=seed + 1)
    _, E_or = ite.full_ite(geom, t, 16, dts, em)
    ctx = P.bbp_create_peps(P.SQUARE, geom_args[0], geom_args[1], 0, 2, 2, t)
    try:
        P.bbp_partition_blocks(ctx, geom_args[2], geom_args[3])
        P.bbp_set_options(ctx, 16, P.FP64)
        P.bbp_init_messages(ctx, em)
        gates = [ite.gate(ite.heisenberg_h(), 0.5 * dt) for dt in dts]
        bonds = [(g1, k1) for (g1, k1, _, _) in geom.bonds()]
        E = P.bbp_ite(ctx, gates, bonds, bp_tol=1e-10, bp_max_iter=40, als_sweeps=50)
    finally:
        P.bbp_destroy(ctx)
    return E, np.array([e.real for e in E_or])


def test_full_ite_two_spins_reach_the_singlet():
    E, E_or = _full((2, 1, 2, 1), [0.5] * 40)
    assert np.max(np.abs(E - E_or)) < 1e-9
    assert abs(E[-1] - (-0.375)) < 1e-8
    print(f"full ITE, two spins: E/site {E[-1]:.12f} (oracle {E_or[-1]:.12f})")


def test_full_ite_three_site_chain():
    E, E_or = _full((3, 1, 3, 1), [0.2] * 20 + [0.05] * 20 + [0.01] * 20)
    assert np.max(np.abs(E - E_or)) < 1e-8
    assert abs(3 * E[-1] - (-1.0)) < 2e-4
    print(f"full ITE, three spins: E {3 * E[-1]:.8f} (oracle {3 * E_or[-1]:.8f}, exact -1)")


def test_full_ite_plaquette_matches_oracle():
    E, E_or = _full((2, 2, 2, 2), [0.2] * 6 + [0.05] * 4)
    assert np.max(np.abs(E - E_or)) < 1e-8
    assert E[-1] < E[0] < 0
    print(f"full ITE, 2 x 2 plaquette: E/site {E[-1]:.8f} (oracle {E_or[-1]:.8f})")


def test_ite_rejects_cross_block_bonds_and_mixed_modes():
    geom, bb, ctx, t = _pair("square", (6, 6, 3, 3), 2, 8, 1, 1)
    G = ite.gate(ite.heisenberg_h(), 0.1)
    try:
        with pytest.raises(P.BBPError) as ei:
            P.bbp_ite_bond(ctx, 2, 1, G)            # site 2 (right column of block 0) -> block 1
        assert ei.value.status == 1
    finally:
        P.bbp_destroy(ctx)
    t = syn.gaussian_peps(36, 2, 2, seed=1)
    ctx = P.bbp_create_peps(P.SQUARE, 6, 6, 0, 2, 2, t)
    try:
        P.bbp_partition_blocks(ctx, 3, 3)
        P.bbp_set_options(ctx, 8, P.TF32)
        P.bbp_init_messages(ctx, syn.initial_edge_matrices(36, 2, seed=2))
        with pytest.raises(P.BBPError) as ei:       # the ITE update runs in the FP64 mode only
            P.bbp_ite_bond(ctx, 7, 1, G)
        assert ei.value.status == 1
    finally:
        P.bbp_destroy(ctx)
