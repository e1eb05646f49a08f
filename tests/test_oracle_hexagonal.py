"""Pins of the oracle's hexagonal Kagome blocks (Sec. 2.3.1, Sec. 2.3 "Contraction Order").

No GPU.  The counts the thesis states for the hexagonal block
(tests/golden/paper_values.json), the tiling rules of Sec. 2.2.2, the six
contraction orders against a brute-force contraction of the block with its
messages, and states on which BlockBP is exact (products and dimer
coverings of singlets).
"""
import json
import math
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import exact, tn
from oracle.hexagonal import HexBlockBP, HexGeometry, _key, _real

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


@pytest.mark.parametrize("N,L", [(2, 7), (3, 19)])
def test_hexagonal_block_counts(N, L):
    """N_T = 3(3N^2 - 3N + 1) (21 and 57); every face carries the same number
    of outgoing edges; for N = 2 the faces alternate 4 and 2 tensors (sites
    on the face line: the extreme depth along its outward normal)."""
    g = HexGeometry(N, L, L)
    assert all(len(b.sites) == GOLDEN["kagome_hexagonal_sites"][str(N)] for b in g.blocks)
    for b in g.blocks:
        counts = {len(b.faces[f].edges) for f in range(6)}
        assert len(counts) == 1 and GOLDEN["kagome_hexagonal_equal_face_edges"]["value"]
        on_face = []
        for f in range(6):
            ks = [_key(f, p)[0] for p in b.pos4]
            on_face.append(sum(1 for k in ks if k == max(ks)))
        if N == 2:
            big, small = GOLDEN["kagome_hexagonal_face_tensors_N2"]["value"]
            assert on_face == [big, small] * 3


@pytest.mark.parametrize("N,Lx,Ly", [(2, 7, 7), (2, 14, 7), (3, 19, 19)])
def test_hexagonal_tiling_rules(N, Lx, Ly):
    """Sec. 2.2.2: the blocks partition the sites; each face borders one
    block, six different ones; the edges of a face enter the opposite face
    of that block, edge for edge in the shared canonical order."""
    g = HexGeometry(N, Lx, Ly)
    seen = [b.gids for b in g.blocks]
    flat = sorted(x for s in seen for x in s)
    assert flat == list(range(g.n_sites))
    for b in g.blocks:
        nbrs = [b.faces[f].nbr for f in range(6)]
        if len(g.blocks) >= 7:
            assert len(set(nbrs)) == 6
        for f in range(6):
            mine = b.faces[f].edges
            other = g.blocks[b.faces[f].nbr].faces[(f + 3) % 6].edges
            assert len(mine) == len(other)
            for e, o in zip(mine, other):
                assert g.blocks[b.faces[f].nbr].gids[o.site] == e.gid and o.slot == e.gslot
                assert b.gids[e.site] == o.gid and e.slot == o.gslot


def _brute_block(bb, b):
    """The block's fused tensors and its six incoming messages, contracted by
    labels without any sweep or truncation (independent of the contraction
    orders), the tensors taken bottom-up by position so that the
    intermediate stays one row wide."""
    g = bb.geom
    blk = g.blocks[b]
    lat = g.lattice
    idx = {s: q for q, s in enumerate(blk.sites)}
    items = []
    for q, (t, i, j) in enumerate(blk.sites):
        labels = []
        for k in range(4):
            t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
            if (t2, i2, j2) in idx:
                labels.append(("i",) + tuple(sorted(((q, k), (idx[(t2, i2, j2)], k2)))))
            else:
                labels.append(("x", q, k))
        x, y = _real(blk.pos4[q])
        items.append(((round(y, 9), round(x, 9)), bb.T[blk.gids[q]], labels))
    for f in range(6):
        mps = bb.msgs[(b, f)]
        K = len(mps)
        for q, (a, e) in enumerate(zip(mps, blk.faces[f].edges)):
            lab = [("m", f, q), ("x", e.site, e.slot), ("m", f, q + 1)]
            X = np.asarray(a)
            if q == 0:
                X, lab = X[0], lab[1:]
            if q == K - 1:
                X, lab = X[..., 0], lab[:-1]
            x, y = _real(e.mid4)
            items.append(((round(y, 9), round(x, 9)), X, lab))
    items.sort(key=lambda z: z[0])
    return exact.contract_network([(X, lab) for _, X, lab in items])


def test_six_contraction_orders_equal_brute_force():
    """The block contracted with its messages towards each of its six faces
    (Sec. 2.3: every direction has its own order) gives the same value, equal
    to the plain contraction of the block with all six messages, when chi
    exceeds every rank."""
    g = HexGeometry(2, 7, 7)
    n = g.n_sites
    bb = HexBlockBP(g, syn.gaussian_peps(n, 2, 2, seed=3), chi=4096)
    bb.init_messages(syn.initial_edge_matrices(n, 2, seed=4))
    bb.step()                                # messages of bond > 1
    for b in (0, 3):
        ref = _brute_block(bb, b)
        for f in range(6):
            ls, z = bb.contract(b, towards=f)
            assert abs(z * math.exp(ls) - ref) < 1e-11 * abs(ref), (b, f)


def test_product_state_hexagonal():
    """D = 1: every message is trivial after one iteration and <S^z> is the
    single-site value."""
    g = HexGeometry(2, 7, 7)
    n = g.n_sites
    t = syn.gaussian_peps(n, 2, 1, seed=5)
    bb = HexBlockBP(g, t, chi=4)
    bb.init_messages(syn.initial_edge_matrices(n, 1, seed=6))
    bb.step()
    assert bb.step() < 1e-13
    for q in (0, 7, 20):
        g0 = g.blocks[2].gids[q]
        v = t[g0][:, 0, 0, 0, 0]
        want = (np.conj(v) @ SZ @ v) / (np.conj(v) @ v)
        assert abs(bb.expect(2, {q: SZ}) - want) < 1e-13


def test_dimer_covering_hexagonal():
    """A product of singlets on a random dimer covering of the 14 x 7 Kagome
    super-cell: BlockBP on hexagonal blocks is exact, every dimer bond inside
    a block has <S.S> = -3/4, every other bond 0, every <S^z> 0."""
    g = HexGeometry(2, 14, 7)
    nb = syn.kagome_neighbours(14, 7)
    t = syn.dimer_singlet_peps(nb, 2, 2, seed=8, noise=0.0, noise_seed=9)
    partner = syn.random_dimer_covering(nb, 8)
    bb = HexBlockBP(g, t, chi=8)
    bb.init_messages(syn.initial_edge_matrices(g.n_sites, 2, seed=10))
    bb.run(1e-12, 6)
    blk = g.blocks[0]
    local = {gg: q for q, gg in enumerate(blk.gids)}
    n_dimer = 0
    for q, gg in enumerate(blk.gids):
        assert abs(bb.expect(0, {q: SZ})) < 1e-12
        for k in range(4):
            g2, k2 = nb[gg][k]
            if g2 not in local or (gg, k) > (g2, k2):
                continue
            e = sum(bb.expect(0, {q: S, local[g2]: S}) for S in (SX, SY, SZ))
            if partner[gg][0] == g2:
                n_dimer += 1
                assert abs(e + 0.75) < 1e-12
            else:
                assert abs(e) < 1e-12
    assert n_dimer > 0


def _hex_env(chi=4096):
    from oracle.hexagonal import HexBlockBP
    g = HexGeometry(2, 7, 7)
    n = g.n_sites
    bb = HexBlockBP(g, syn.gaussian_peps(n, 2, 2, seed=3), chi=chi)
    bb.init_messages(syn.initial_edge_matrices(n, 2, seed=4))
    bb.step()
    return g, bb


def test_hexagonal_core_route_is_exact():
    """Sec. 2.3, Core, in the hexagonal block: two bubbles from the D and U
    faces around a core, joined by the zipper, give exactly the block's value
    with operators on the core (chi above every rank): one site, a bond, the
    centre unit cell, three unit cells."""
    from oracle.hexagonal import HexCoreEnv
    g, bb = _hex_env()
    b = g.blocks[0]
    ci, cj = b.centre

    def cell(i, j):
        return [b.sites.index((t, ci + i, cj + j)) for t in (2, 0, 1)]

    for core in (cell(0, 0)[:1], cell(0, 0)[:2], cell(0, 0), cell(0, 0) + cell(1, 0) + cell(1, -1)):
        env = HexCoreEnv(bb, 0, core)
        for q in core[:3]:
            assert abs(env.expect({q: SZ}) - bb.expect(0, {q: SZ})) < 1e-12


def test_hexagonal_core_of_three_cells_and_its_modes():
    """The core of three unit cells around a down-triangle (Sec. 2.3, Core,
    Modes): the three up-triangle bond types appear three times and the three
    down-triangle types once; it holds three modes (an up-triangle and the
    shared down-triangle), each holding every one of the six bond types
    once; from a mode the Edge TN of each of its bonds follows by exact
    contraction and gives the bond's RDM."""
    from oracle import core as C
    from oracle.hexagonal import HexCoreEnv
    g, bb = _hex_env()
    lat = g.lattice
    b = g.blocks[0]
    ci, cj = b.centre
    cells = [(ci, cj), (ci + 1, cj), (ci + 1, cj - 1)]
    core = [b.sites.index((t, i, j)) for (i, j) in cells for t in range(3)]
    env = HexCoreEnv(bb, 0, core)
    count = {}
    for x in range(len(core)):
        for y in range(x + 1, len(core)):
            shared = set(env.sites[core[x]].labels) & set(env.sites[core[y]].labels)
            for lab in shared:
                s = env.sites[core[x]].labels.index(lab)
                ty = C.bond_type(lat, b.sites[core[x]][0], s)
                count[ty] = count.get(ty, 0) + 1
    ref = GOLDEN["kagome_core_three_cells"]
    assert sorted(count.values()) == ref["bond_multiplicities"]
    modes = [C.kagome_mode(g, 0, cells[0], 1), C.kagome_mode(g, 0, cells[1], 0), C.kagome_mode(g, 0, cells[2], 2)]
    assert len(modes) == ref["modes"]
    for mode in modes:
        assert mode is not None and set(mode) <= set(core)
        types = set()
        for x in range(5):
            for y in range(x + 1, 5):
                shared = set(env.sites[mode[x]].labels) & set(env.sites[mode[y]].labels)
                for lab in shared:
                    types.add(C.bond_type(lat, b.sites[mode[x]][0], env.sites[mode[x]].labels.index(lab)))
        assert len(types) == ref["bond_types_per_mode"]
    mode = modes[0]
    menv = HexCoreEnv(bb, 0, mode)
    k1, k2 = mode[0], mode[1]
    N, _, slots = menv.edge(k1, k2)
    r1, r2 = menv.sites[k1], menv.sites[k2]
    jt = next(iter(set(r1.labels) & set(r2.labels)))
    rho = C.edge_rdm(N, slots, 2, 2, 2, bb.tc[r1.gid], bb.tc[r2.gid], r1.labels.index(jt), r2.labels.index(jt))
    direct = HexCoreEnv(bb, 0, [k1, k2]).rdm([k1, k2])
    assert np.abs(rho - direct).max() < 1e-12
