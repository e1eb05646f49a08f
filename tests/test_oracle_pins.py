"""Pins of the FP64 oracle against what the thesis and the mathematics fix.

No GPU.  Each test ties one part of the oracle to something other than the
oracle itself: a closed form, brute force, an independent restatement, or a
value the thesis prints (tests/golden/paper_values.json).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import exact, tn
from oracle.blockbp import BlockBP, message_distance, normalise_message
from oracle.bp import SiteBP
from oracle.geometry import BOTTOM, LEFT, RIGHT, TOP, Geometry

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


# ------------------------------------------------------------------ fusion --

def test_fuse_matches_definition_by_loops():
    """T[(u u'),(r r'),(d d'),(l l')] = sum_s t[s,u,r,d,l] conj(t[s,u',r',d',l'])
    written out with explicit loops (Sec. 2.1)."""
    rng = np.random.default_rng(0)
    d, D = 2, 2
    t = rng.standard_normal((d, D, D, D, D)) + 1j * rng.standard_normal((d, D, D, D, D))
    T = tn.fuse(t)
    for legs in itertools.product(range(D), repeat=8):
        k = legs[0::2]
        b = legs[1::2]
        ref = sum(t[(s,) + k] * np.conj(t[(s,) + b]) for s in range(d))
        idx = tuple(k[q] * D + b[q] for q in range(4))
        assert abs(T[idx] - ref) < 1e-14


def test_fuse_hermitian_and_psd():
    rng = np.random.default_rng(1)
    d, D = 2, 3
    t = rng.standard_normal((d, D, D, D, D)) + 1j * rng.standard_normal((d, D, D, D, D))
    T = tn.fuse(t).reshape([D] * 8)
    # swapping ket <-> bra on every leg at once conjugates T
    Tsw = T.transpose(1, 0, 3, 2, 5, 4, 7, 6)
    assert np.allclose(Tsw, np.conj(T), atol=1e-13)
    # as a matrix [(ket legs), (bra legs)] it is sum_s v_s v_s^dagger: PSD, rank <= d
    M = T.transpose(0, 2, 4, 6, 1, 3, 5, 7).reshape(D ** 4, D ** 4)
    w = np.linalg.eigvalsh(M)
    assert w.min() > -1e-10 * w.max()
    assert np.sum(w > 1e-10 * w.max()) <= d


def test_fuse_operator_single_site_closed_form():
    """With D = 1 the fused tensor is the number <t|O|t>."""
    rng = np.random.default_rng(2)
    v = rng.standard_normal(2) + 1j * rng.standard_normal(2)
    t = v.reshape(2, 1, 1, 1, 1)
    for O in (SX, SY, SZ):
        val = tn.fuse(t, O).reshape(())
        assert abs(val - np.vdot(v, O @ v)) < 1e-14


# ------------------------------------------------------ SVD and MPS pieces --

def test_svd_split_eckart_young():
    rng = np.random.default_rng(3)
    m, n, chi = 12, 9, 4
    U, _ = np.linalg.qr(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    s = np.array([5.0, 3.0, 2.0, 1.5, 1.0, 0.5, 0.25, 0.125, 0.0625])
    M = (U * s) @ V.conj().T
    R = M.reshape(3, 4, 9)              # (l, q1, rest) with rest = (q2, r)
    A1, rem = tn.svd_split(R.reshape(3, 4, 3, 3), chi)
    approx = np.tensordot(A1, rem, axes=(2, 0)).reshape(m, n)
    assert A1.shape[2] == chi
    err = np.linalg.norm(M - approx)
    assert abs(err - math.sqrt(np.sum(s[chi:] ** 2))) < 1e-12
    got = np.linalg.svd(approx, compute_uv=False)[:chi]
    assert np.allclose(got, s[:chi], atol=1e-12)


def _random_mps(rng, dims, chi):
    A = []
    l = 1
    for q, p in enumerate(dims):
        r = 1 if q == len(dims) - 1 else chi
        A.append(rng.standard_normal((l, p, r)) + 1j * rng.standard_normal((l, p, r)))
        l = r
    return A


def test_distance_and_normalisation_dense():
    rng = np.random.default_rng(4)
    dims = [4, 4, 4]
    a = normalise_message(_random_mps(rng, dims, 3), [2, 2, 2])
    b = normalise_message(_random_mps(rng, dims, 3), [2, 2, 2])
    va, vb = tn.mps_dense(a), tn.mps_dense(b)
    assert abs(np.vdot(va, va) - 1) < 1e-13
    idv = np.zeros(64)
    for k in itertools.product(range(2), repeat=3):
        idv[np.ravel_multi_index([kk * 2 + kk for kk in k], dims)] = 1
    tr = np.vdot(idv, va)
    assert tr.real > 0 and abs(tr.imag) < 1e-13
    assert abs(message_distance(a, b) - np.linalg.norm(va - vb)) < 1e-13
    # resolves tiny distances (no sqrt(2 - 2 Re<a|b>) cancellation floor)
    c = [x.copy() for x in a]
    c[1] = c[1] + 1e-12 * rng.standard_normal(c[1].shape)
    exact_d = np.linalg.norm(tn.mps_dense(c) - va)
    assert abs(message_distance(a, c) - exact_d) < 1e-15


def test_canonical_moves_preserve_state_and_isometry():
    rng = np.random.default_rng(5)
    A = _random_mps(rng, [3, 5, 4], 4)
    v0 = tn.mps_dense(A)
    Q, B = tn.qr_right(A[0], A[1])
    v1 = tn.mps_dense([Q, B, A[2]])
    assert np.allclose(v0, v1, atol=1e-12)
    q = Q.reshape(-1, Q.shape[2])
    assert np.allclose(q.conj().T @ q, np.eye(q.shape[1]), atol=1e-13)
    C, Q2 = tn.lq_left(A[1], A[2])
    v2 = tn.mps_dense([A[0], C, Q2])
    assert np.allclose(v0, v2, atol=1e-12)
    q2 = Q2.reshape(Q2.shape[0], -1)
    assert np.allclose(q2 @ q2.conj().T, np.eye(q2.shape[0]), atol=1e-13)


# ------------------------------------------------------------ exact / sweep --

def test_exact_contraction_vs_full_einsum():
    """The sweep-line brute force equals one einsum of all four tensors (2 x 2)."""
    geom = Geometry.square(2, 2, 2, 2)
    t = syn.gaussian_peps(4, 2, 3, seed=11)
    T = []
    for g in range(4):
        sl = []
        r, c = divmod(g, 2)
        sl = [slice(None),
              slice(0, 1) if r == 0 else slice(None), slice(0, 1) if c == 1 else slice(None),
              slice(0, 1) if r == 1 else slice(None), slice(0, 1) if c == 0 else slice(None)]
        T.append(tn.fuse(t[g][tuple(sl)]).squeeze())
    # legs kept: site 0 (top-left) [r, d]; site 1 [d, l]; site 2 [u, r]; site 3 [u, l]
    z = np.einsum("ab,ca,bd,cd->", T[0], T[1], T[2], T[3])
    assert abs(z - exact.norm(geom.lattice, t)) < 1e-12 * abs(z)


@pytest.mark.parametrize("shape", [(3, 3, 2), (2, 3, 3), (3, 2, 2)])
def test_single_block_sweep_equals_exact(shape):
    """A block covering the whole open lattice with chi above every rank:
    the boundary-MPS sweep is exact (no truncation), for any out face."""
    Lx, Ly, D = shape
    geom = Geometry.square(Lx, Ly, Lx, Ly)
    t = syn.gaussian_peps(Lx * Ly, 2, D, seed=12)
    bb = BlockBP(geom, t, chi=10 ** 4)
    zex = exact.norm(geom.lattice, t)
    l, z = bb.contract([(0, 0)])
    assert abs(z * math.exp(l) - zex) < 1e-11 * abs(zex)
    for g in range(Lx * Ly):
        ref = exact.expect(geom.lattice, t, {g: SZ})
        got = bb.sz(g)
        assert abs(got - ref) < 1e-11


def test_truncation_error_decreases_with_chi():
    """Truncated sweeps approach the exact value as chi grows (Sec. 1.1.3)."""
    geom = Geometry.square(4, 4, 4, 4)
    t = syn.gaussian_peps(16, 2, 2, seed=13)
    zex = exact.norm(geom.lattice, t)
    errs = []
    for chi in (2, 4, 16, 64):
        bb = BlockBP(geom, t, chi=chi)
        l, z = bb.contract([(0, 0)])
        errs.append(abs(z * math.exp(l) - zex) / abs(zex))
    assert errs[-1] < 1e-12
    assert errs[0] > errs[-1]


# ------------------------------------------------------------- BlockBP pins --

def test_blockbp_1x1_blocks_reduce_to_bp():
    """Blocks of one site: every message is a single D x D matrix and the
    update is exactly Eq. of BP (Sec. 2.1), restated independently in bp.py."""
    geom = Geometry.square(3, 3, 1, 1)
    t = syn.gaussian_peps(9, 2, 2, seed=21)
    em = syn.initial_edge_matrices(9, 2, seed=22)
    bb = BlockBP(geom, t, chi=64)
    bb.init_messages(em)
    sbp = SiteBP(geom.lattice, t)
    sbp.init(em)
    for _ in range(4):
        e1 = bb.step()
        e2 = sbp.step()
        assert abs(e1 - e2) < 1e-12
        for (bid, d), m in bb.msgs.items():
            blk = geom.blocks[bid]
            e = blk.faces[d].edges[0]
            assert np.abs(tn.mps_dense(m) - sbp.m[(blk.gids[e.site], e.slot)]).max() < 1e-13


@pytest.mark.parametrize("layout", [(6, 2, 2, 2), (2, 6, 2, 2), (6, 3, 2, 3)])
def test_tree_of_blocks_is_exact(layout):
    """A chain of blocks has no loops between blocks, so BlockBP with chi above
    every rank is exact (Sec. 2.1): observables and the Bethe log-norm equal
    brute force, and the iteration reaches a fixed point."""
    Lx, Ly, bx, by = layout
    geom = Geometry.square(Lx, Ly, bx, by)
    n = Lx * Ly
    t = syn.gaussian_peps(n, 2, 2, seed=31)
    bb = BlockBP(geom, t, chi=512)
    bb.init_messages(syn.initial_edge_matrices(n, 2, seed=32))
    it, err = bb.run(1e-13, 12)
    assert err < 1e-13
    for g in range(n):
        assert abs(bb.sz(g) - exact.expect(geom.lattice, t, {g: SZ})) < 1e-11
    for (g1, k1, g2, k2) in geom.bonds():
        ref = sum(exact.expect(geom.lattice, t, {g1: O, g2: O}) for O in (SX, SY, SZ))
        assert abs(bb.heisenberg_bond(g1, k1) - ref) < 1e-11
    assert abs(bb.log_norm() - math.log(abs(exact.norm(geom.lattice, t)))) < 1e-10


def test_product_state_converges_in_one_iteration():
    """D = 1: the network is a product, every message is trivial after one
    update and <S^z> is the single-site value exactly."""
    geom = Geometry.square(4, 4, 2, 2)
    rng = np.random.default_rng(41)
    v = rng.standard_normal((16, 2)) + 1j * rng.standard_normal((16, 2))
    t = v.reshape(16, 2, 1, 1, 1, 1)
    bb = BlockBP(geom, t, chi=4)
    bb.init_messages(syn.initial_edge_matrices(16, 1, seed=42))
    bb.step()
    assert bb.step() < 1e-14
    for g in range(16):
        ref = np.vdot(v[g], SZ @ v[g]) / np.vdot(v[g], v[g])
        assert abs(bb.sz(g) - ref) < 1e-13


def test_two_spin_singlet_energy():
    """1 x 2 PEPS carrying (|01> - |10>)/sqrt 2 through a D = 2 bond:
    <S1.S2> = -3/4 (Eq. of the AFM Heisenberg Hamiltonian)."""
    geom = Geometry.square(2, 1, 1, 1)
    nb = syn.square_neighbours(2, 1, False)
    t = syn.dimer_singlet_peps(nb, 2, 2, seed=0, noise=0.0, noise_seed=0)
    bb = BlockBP(geom, t, chi=4)
    bb.init_messages(syn.initial_edge_matrices(2, 2, seed=51))
    bb.run(1e-14, 5)
    e = bb.heisenberg_bond(0, 1)
    assert abs(e - GOLDEN["heisenberg_singlet_bond_energy"]["value"]) < 1e-13


@pytest.mark.parametrize("lat", ["square", "kagome"])
def test_dimer_covering_is_exact(lat):
    """A product of singlets on a perfect dimer covering: the virtual graph is
    a forest, so BlockBP is exact: -3/4 on dimer bonds, 0 on all others
    (Kagome: energy per site -3/8)."""
    if lat == "square":
        geom = Geometry.square(4, 4, 2, 2, periodic=True)
        nb = syn.square_neighbours(4, 4, True)
    else:
        geom = Geometry.kagome(6, 2, 2)
        nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, 2, seed=2, noise=0.0, noise_seed=0)
    partner = syn.random_dimer_covering(nb, 2)
    bb = BlockBP(geom, t, chi=8)
    bb.init_messages(syn.initial_edge_matrices(geom.n_sites, 2, seed=52))
    bb.run(1e-13, 6)
    for (g1, k1, g2, k2) in geom.bonds():
        e = bb.heisenberg_bond(g1, k1)
        want = -0.75 if (partner[g1][0] == g2 and partner[g1][1] == k1) else 0.0
        assert abs(e - want) < 1e-12
    if lat == "kagome":
        assert abs(bb.energy_per_site() + 0.375) < 1e-12


def test_rdm_tree_exact_and_physical():
    geom = Geometry.square(6, 2, 2, 2)
    t = syn.gaussian_peps(12, 2, 2, seed=61)
    bb = BlockBP(geom, t, chi=512)
    bb.init_messages(syn.initial_edge_matrices(12, 2, seed=62))
    bb.run(1e-13, 10)
    coords, k1, k2 = bb.bond_region(1, 1)     # site 1 and its right neighbour (site 2, next block)
    rho = bb.rdm([k1, k2], coords)
    ref = exact.rdm(geom.lattice, t, [1, 2])
    ref = ref / np.trace(ref)
    assert np.abs(rho - ref).max() < 1e-11
    assert np.allclose(rho, rho.conj().T, atol=1e-12)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.linalg.eigvalsh((rho + rho.conj().T) / 2).min() > -1e-12


def test_rdm_loopy_physical():
    geom = Geometry.square(4, 4, 2, 2)
    t = syn.gaussian_peps(16, 2, 2, seed=71)
    bb = BlockBP(geom, t, chi=8)
    bb.init_messages(syn.initial_edge_matrices(16, 2, seed=72))
    bb.run(1e-10, 30)
    b, loc = bb.home(5)
    rho = bb.rdm([(0, loc)], [(b.X, b.Y)])
    assert np.allclose(rho, rho.conj().T, atol=1e-10)
    assert np.linalg.eigvalsh((rho + rho.conj().T) / 2).min() > -1e-8
    for (g1, k1, g2, k2) in geom.bonds()[:6]:
        e = bb.heisenberg_bond(g1, k1).real
        assert -0.75 - 1e-8 <= e <= 0.25 + 1e-8


# ---------------------------------------------------------------- geometry --

@pytest.mark.parametrize("L", [2, 3, 4])
def test_kagome_parallelogram_counts(L):
    geom = Geometry.kagome(3 * L, L, L)
    want = GOLDEN["kagome_parallelogram_sites"][str(L)]
    for b in geom.blocks:
        assert len(b.sites) == want == 3 * L * L
        counts = [len(b.faces[d].edges) for d in range(4)]
        assert counts[BOTTOM] == counts[TOP] and counts[LEFT] == counts[RIGHT]
        assert counts == [2 * L] * 4
    # the blocks tile the super-cell: every site exactly once
    all_ids = sorted(g for b in geom.blocks for g in b.gids)
    assert all_ids == list(range(geom.n_sites))
    # four legs per site: 2 * internal + crossing = 4 N_T
    for b in geom.blocks:
        crossing = sum(len(b.faces[d].edges) for d in range(4))
        assert 2 * len(b.internal) + crossing == 4 * len(b.sites)


def test_kagome_faces_match_across_blocks():
    """Every crossing bond of face d enters the opposite face of the neighbour
    (Sec. 2.2.2), with the same canonical order seen from both sides."""
    geom = Geometry.kagome(6, 2, 2)
    for b in geom.blocks:
        for d in range(4):
            f = b.faces[d]
            g = geom.blocks[f.nbr].faces[(d + 2) % 4]
            mine = [(b.gids[e.site], e.slot, e.gid, e.gslot) for e in f.edges]
            theirs = [(e.gid, e.gslot, geom.blocks[f.nbr].gids[e.site], e.slot) for e in g.edges]
            assert mine == theirs


def test_square_blocks():
    geom = Geometry.square(6, 6, 3, 3)
    assert len(geom.blocks) == 4
    assert len(geom.updates()) == 8
    for b in geom.blocks:
        assert len(b.sites) == 9
        assert sorted(len(b.faces[d].edges) for d in range(4)) == [3, 3, 3, 3]


@pytest.mark.parametrize("L", [2, 3])
def test_translation_invariant_kagome_gives_equal_block_messages(L):
    """With the same three site tensors in every unit cell and the same
    initial edge matrices in every cell, a translation by L unit cells maps
    every block of the 3L x L super-cell onto the next one (Sec. 2.3.1,
    periodic super-cell): after any number of synchronous iterations each
    face of every block carries the same message.  A wrong periodic
    neighbour, face or re-homed corner site breaks the equality."""
    Lx, Ly, D = 3 * L, L, 2
    n = 3 * Lx * Ly
    cell = syn.gaussian_peps(3, 2, D, seed=41)
    t = np.stack([cell[s % 3] for s in range(n)])
    em_cell = syn.initial_edge_matrices(3, D, seed=42)
    em = np.stack([em_cell[s % 3] for s in range(n)])
    geom = Geometry.kagome(Lx, Ly, L)
    assert len(geom.blocks) == 3
    bb = BlockBP(geom, t, chi=4)
    bb.init_messages(em)
    for _ in range(2):
        bb.step()
    for face in range(4):
        dense = [tn.mps_dense(bb.msgs[(b, face)]) for b in range(3) if (b, face) in bb.msgs]
        assert len(dense) == 3
        for other in dense[1:]:
            assert np.abs(other - dense[0]).max() < 1e-12
