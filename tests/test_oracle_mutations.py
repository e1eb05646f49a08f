"""Planted mistakes in the oracle (CPU only): each must be caught by a pin.

A pin that cannot fail proves nothing; these tests plant plausible errors
(a transposed leg order, an off-by-one truncation) in
the oracle and check that the comparison against brute force notices.
"""
import math

import numpy as np

import synthetic as syn
from oracle import exact, tn
from oracle.blockbp import BlockBP
from oracle.geometry import Geometry


def _single_block_error(monkeypatch_ctx=None, chi=10 ** 4, D=2):
    geom = Geometry.square(3, 3, 3, 3)
    t = syn.gaussian_peps(9, 2, D, seed=12)
    bb = BlockBP(geom, t, chi=chi)
    zex = exact.norm(geom.lattice, t)
    try:
        l, z = bb.contract([(0, 0)])
    except Exception:
        return math.inf
    return abs(z * math.exp(l) - zex) / abs(zex)


def test_clean_oracle_is_exact():
    assert _single_block_error() < 1e-12


def test_out_leg_order_flip_is_caught(monkeypatch):
    real_transpose = np.transpose
    calls = {"n": 0}

    def bad_transpose(a, axes=None):
        # reverse the out-leg order of every swallowed site tensor (4 legs)
        if axes is not None and len(axes) == 4 and a.ndim == 4:
            calls["n"] += 1
            axes = list(axes)
            nin = 2
            axes = axes[:nin] + axes[nin:][::-1]
        return real_transpose(a, axes)
    monkeypatch.setattr(tn.np, "transpose", bad_transpose)
    assert _single_block_error() > 1e-6
    assert calls["n"] > 0


def test_truncation_off_by_one_is_caught(monkeypatch):
    real = tn.svd_split

    def bad_split(R, chi):
        sh = R.shape
        M = R.reshape(sh[0] * sh[1], -1)
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        k = max(1, min(chi, M.shape[0], M.shape[1]) - 1)    # keeps one too few
        return U[:, :k].reshape(sh[0], sh[1], k), (s[:k, None] * Vh[:k]).reshape((k,) + sh[2:])
    monkeypatch.setattr(tn, "svd_split", bad_split)
    assert _single_block_error() > 1e-8
    monkeypatch.setattr(tn, "svd_split", real)


def test_zipper_front_line_transposed_is_caught(monkeypatch):
    """Plant a transposed left front-line matrix in the core's zipper: the
    core route on a tree of blocks must then miss the brute-force <S^z>."""
    from oracle import core as C
    geom = Geometry.square(6, 3, 3, 3)
    t = syn.gaussian_peps(18, 2, 2, seed=41)
    bb = BlockBP(geom, t, chi=512)
    bb.init_messages(syn.initial_edge_matrices(18, 2, seed=42))
    bb.run(1e-13, 12)
    sz = np.diag([0.5, -0.5]).astype(np.complex128)
    b = geom.blocks[0]
    ref = exact.expect(geom.lattice, t, {b.gids[4]: sz})
    env = C.CoreEnv(bb, [(b.X, b.Y)], [(0, 4)])
    assert abs(env.expect({(0, 4): sz}) - ref) < 1e-12
    real_einsum = C.np.einsum

    def bad_einsum(spec, *ops, **kw):
        if spec == "xy,xpz,wpy->zw":
            spec = "xy,xpz,wpy->wz"
        return real_einsum(spec, *ops, **kw)
    monkeypatch.setattr(C.np, "einsum", bad_einsum)
    try:
        err = abs(C.CoreEnv(bb, [(b.X, b.Y)], [(0, 4)]).expect({(0, 4): sz}) - ref)
    except Exception:
        err = math.inf
    assert err > 1e-6


def test_ite_gate_sign_flip_is_caught(monkeypatch):
    """Plant exp(+dt h) for exp(-dt h) in the ITE oracle: the two-spin run
    must then miss the singlet energy the pin fixes."""
    from oracle import ite
    real_gate = ite.gate
    geom = Geometry.square(2, 1, 2, 1)
    t = syn.gaussian_peps(2, 2, 2, seed=13)
    em = syn.initial_edge_matrices(2, 2, seed=14)
    _, E = ite.full_ite(geom, t, 16, [0.5] * 20, em)
    assert abs(E[-1].real + 0.375) < 1e-6
    monkeypatch.setattr(ite, "gate", lambda h, dt: real_gate(h, -dt))
    _, E = ite.full_ite(geom, t, 16, [0.5] * 20, em)
    assert abs(E[-1].real + 0.375) > 0.1


def test_hexagonal_face_order_flip_is_caught(monkeypatch):
    """Plant a reversed canonical edge order on one face of the hexagonal
    blocks: the edge-for-edge pairing of opposite faces must then fail."""
    from oracle import hexagonal as H
    real = H._canon
    monkeypatch.setattr(H, "_canon", lambda f, p4: -real(f, p4) if f == 1 else real(f, p4))
    g = H.HexGeometry(2, 7, 7)
    bad = 0
    for b in g.blocks:
        mine = b.faces[1].edges
        other = g.blocks[b.faces[1].nbr].faces[4].edges
        bad += sum(1 for e, o in zip(mine, other) if g.blocks[b.faces[1].nbr].gids[o.site] != e.gid)
    assert bad > 0
