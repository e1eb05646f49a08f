"""Core extraction on the GPU (bbp_core_pmps) against the oracle (Sec. 2.3, "Core").

The GPU's two bubbles and zipper leave a periodic MPS (pMPS) around the
core.  Its tensors carry SVD and QR gauges, so the test contracts the GPU's
pMPS with the oracle's fused core tensors and compares gauge-invariant
numbers with the oracle's own core route on the same messages (both sides
iterate the same seeded network first): <S^z> of every core site, a bond
energy inside the core, and the log of the core's value (log scale plus
log |Z|).  FP64 mode: 1e-10; TF32 mode (complex64 bubbles): 1e-5.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import core as C
from oracle import exact
from oracle.blockbp import BlockBP
from oracle.geometry import Geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")

SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def _pair(kind, args, D, chi, iters, seed, precision):
    if kind == "square":
        geom = Geometry.square(*args)
    else:
        geom = Geometry.kagome(*args)
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
    P.bbp_set_options(ctx, chi, precision)
    P.bbp_init_messages(ctx, em)
    it, _, _ = P.bbp_iterate(ctx, 0.0, iters)
    assert it == iters
    return geom, bb, ctx


def _gpu_value(env, ring, legs, ops=None):
    """The GPU pMPS closed with the oracle's core tensors (operators inserted)."""
    L = len(ring)
    items = []
    for q, (X, (k, slot)) in enumerate(zip(ring, legs)):
        lab = env.sites[env.core[k]].labels[slot]
        items.append((X, [("ring", q), lab, ("ring", (q + 1) % L)]))
    return exact.contract_network(items + env.core_items(ops))


def _check(geom, bb, ctx, block, core_locals, tol):
    b = geom.blocks[block]
    keys = [(0, q) for q in core_locals]
    env = C.CoreEnv(bb, [(b.X, b.Y)], keys)
    ring, legs, ls = P.bbp_core_pmps(ctx, block, [b.gids[q] for q in core_locals])
    assert len(ring) == len(env.pmps)
    for q in range(len(ring)):                       # the ring closes
        assert ring[q].shape[2] == ring[(q + 1) % len(ring)].shape[0]
    z0 = _gpu_value(env, ring, legs)
    lz_gpu = ls + math.log(abs(z0))
    l0, zo = env.value()
    lz_or = l0 + math.log(abs(zo))
    assert abs(lz_gpu - lz_or) < tol * max(1.0, abs(lz_or)), (lz_gpu, lz_or)
    worst = 0.0
    for k in keys:
        e_gpu = _gpu_value(env, ring, legs, {k: SZ}) / z0
        worst = max(worst, abs(e_gpu - env.expect({k: SZ})))
    if len(keys) >= 2:
        k1, k2 = keys[0], keys[1]
        if set(env.sites[k1].labels) & set(env.sites[k2].labels):
            e_gpu = sum(_gpu_value(env, ring, legs, {k1: S, k2: S}) for S in (SX, SY, SZ)) / z0
            e_or = sum(env.expect({k1: S, k2: S}) for S in (SX, SY, SZ))
            worst = max(worst, abs(e_gpu - e_or))
    assert worst < tol, worst
    return worst


@pytest.mark.parametrize("core_locals", [[4], [3, 4], [1, 4, 5], [4, 7]])
def test_core_pmps_square_fp64(core_locals):
    """6 x 6 open square PEPS (config 1 shape: D = 2, chi = 8, 3 x 3 blocks)
    after three iterations: every block's pMPS around one, two or three
    sites matches the oracle's to 1e-10."""
    geom, bb, ctx = _pair("square", (6, 6, 3, 3), 2, 8, 3, 1, P.FP64)
    try:
        for block in range(len(geom.blocks)):
            w = _check(geom, bb, ctx, block, core_locals, 1e-10)
        print(f"square core {core_locals}: largest observable difference {w:.2e}")
    finally:
        P.bbp_destroy(ctx)


def test_core_pmps_kagome_unit_cell_fp64():
    """Kagome periodic 6 x 2 super-cell, L = 2 blocks, D = 2, chi = 16, two
    iterations: the pMPS around the unit cell (up-triangle A, B, C) of every
    block matches the oracle's to 1e-10 (six open legs, truncating bubbles)."""
    geom, bb, ctx = _pair("kagome", (6, 2, 2), 2, 16, 2, 7, P.FP64)
    try:
        for block in range(len(geom.blocks)):
            b = geom.blocks[block]
            i, j = b.sites[2][1:]
            cell = [b.sites.index((t, i, j)) for t in range(3)]
            w = _check(geom, bb, ctx, block, cell, 1e-10)
        print(f"kagome unit cell: largest observable difference {w:.2e}")
    finally:
        P.bbp_destroy(ctx)


def test_core_pmps_square_tf32():
    """The same extraction in the TF32 mode (complex64 bubbles, split-TF32
    absorb) stays within 1e-5 of the FP64 oracle."""
    geom, bb, ctx = _pair("square", (6, 6, 3, 3), 2, 8, 3, 1, P.TF32)
    try:
        w = _check(geom, bb, ctx, 0, [3, 4], 1e-5)
        print(f"square core TF32: largest observable difference {w:.2e}")
    finally:
        P.bbp_destroy(ctx)


def test_core_pmps_rejects_bad_cores():
    geom, bb, ctx = _pair("square", (6, 6, 3, 3), 2, 8, 1, 1, P.FP64)
    try:
        b = geom.blocks[0]
        other = geom.blocks[1].gids[0]
        with pytest.raises(P.BBPError) as ei:
            P.bbp_core_pmps(ctx, 0, [other])             # not a site of the block
        assert ei.value.status == 1
        with pytest.raises(P.BBPError) as ei:
            P.bbp_core_pmps(ctx, 0, [b.gids[4], b.gids[4]])
        assert ei.value.status == 1
    finally:
        P.bbp_destroy(ctx)


# ----------------------------------------------- local quantities of a core

def _core_checks(geom, bb, ctx, block, cores, tol):
    """bbp_core_expect against the oracle's core route: <S^z> on one-site
    cores, <S^a S^a> (a = x, y, z) on bond cores."""
    b = geom.blocks[block]
    worst = 0.0
    for core in cores:
        keys = [(0, q) for q in core]
        env = C.CoreEnv(bb, [(b.X, b.Y)], keys)
        gids = [b.gids[q] for q in core]
        if len(core) == 1:
            sets = [[SZ], [SX]]
        else:
            sets = [[S, S] for S in (SX, SY, SZ)]
        got = P.bbp_core_expect(ctx, block, gids, sets)
        want = [env.expect({k: o for k, o in zip(keys, ops)}) for ops in sets]
        worst = max(worst, float(np.max(np.abs(np.asarray(got) - np.asarray(want)))))
    assert worst < tol, worst
    return worst


def test_core_expect_square_fp64():
    """One-site cores (a corner, an edge and the centre of each 3 x 3 block)
    and bond cores (horizontal and vertical) of the 6 x 6 square PEPS after
    three iterations: every value equals the oracle's core route to 1e-10."""
    geom, bb, ctx = _pair("square", (6, 6, 3, 3), 2, 8, 3, 1, P.FP64)
    try:
        w = 0.0
        for block in range(len(geom.blocks)):
            w = max(w, _core_checks(geom, bb, ctx, block, [[0], [1], [4], [3, 4], [4, 7], [0, 1]], 1e-10))
        print(f"square core observables FP64: largest difference {w:.2e}")
    finally:
        P.bbp_destroy(ctx)


def test_core_expect_kagome_fp64():
    """Kagome D = 2, chi = 16: every site of each block's first unit cell and
    its three bonds A-B, B-C, C-A (the Edge TN of each) against the oracle."""
    geom, bb, ctx = _pair("kagome", (6, 2, 2), 2, 16, 2, 7, P.FP64)
    try:
        w = 0.0
        for block in range(len(geom.blocks)):
            b = geom.blocks[block]
            i, j = b.sites[2][1:]
            a_, b_, c_ = [b.sites.index((t, i, j)) for t in range(3)]
            w = max(w, _core_checks(geom, bb, ctx, block, [[a_], [b_], [c_], [a_, b_], [b_, c_], [c_, a_]], 1e-10))
        print(f"kagome core observables FP64: largest difference {w:.2e}")
    finally:
        P.bbp_destroy(ctx)


def test_core_expect_tf32():
    geom, bb, ctx = _pair("square", (6, 6, 3, 3), 2, 8, 3, 1, P.TF32)
    try:
        w = _core_checks(geom, bb, ctx, 0, [[4], [3, 4]], 1e-5)
        print(f"square core observables TF32: largest difference {w:.2e}")
    finally:
        P.bbp_destroy(ctx)


def test_core_expect_rejects_bad_cores():
    geom, bb, ctx = _pair("square", (6, 6, 3, 3), 2, 8, 1, 1, P.FP64)
    try:
        b = geom.blocks[0]
        with pytest.raises(P.BBPError) as ei:          # three sites
            P.bbp_core_expect(ctx, 0, [b.gids[q] for q in (3, 4, 5)], [[SZ, SZ, SZ]])
        assert ei.value.status == 1
        with pytest.raises(P.BBPError) as ei:          # two sites that share no bond
            P.bbp_core_expect(ctx, 0, [b.gids[0], b.gids[4]], [[SZ, SZ]])
        assert ei.value.status == 1
    finally:
        P.bbp_destroy(ctx)
