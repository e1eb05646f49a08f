"""Host-side logic of the CUDA library, checked without a GPU.

* the shared library loads and exports every symbol include/bbp.h declares;
* the C++ sweep-plan compiler visits the same nodes, in the same order and
  with the same in/out leg counts, as the oracle's boundary-MPS sweep, for
  every face of several block geometries (two independent implementations of
  the same reading of Sec. 1.1.3 / Sec. 2.3.1);
* argument validation returns error codes instead of crashing.
"""
import os
import re

import numpy as np
import pytest

import synthetic as syn
from oracle.blockbp import BlockBP
from oracle.geometry import Geometry

P = pytest.importorskip("paper_2603_13304_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    P.build()
    return P.lib()


def test_exports_match_header(L):
    hdr = open(os.path.join(ROOT, "include", "bbp.h")).read()
    declared = set(re.findall(r"\b(bbp_[a-z0-9_]+)\s*\(", hdr))
    declared -= {"bbp_alloc_fn", "bbp_free_fn"}
    assert declared == set(P.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


GEOMS = [
    ("square", (6, 6, 3, 3)),
    ("square", (4, 4, 2, 2)),
    ("square", (3, 3, 1, 1)),
    ("square", (6, 4, 3, 2)),
    ("kagome", (6, 2, 2)),
    ("kagome", (9, 3, 3)),
    ("kagome", (4, 4, 4)),
]


@pytest.mark.parametrize("kind,args", GEOMS)
def test_plan_matches_oracle_sweep(L, kind, args):
    if kind == "square":
        geom = Geometry.square(*args)
        lat, Lx, Ly, per, bx, by = 0, args[0], args[1], 0, args[2], args[3]
    else:
        geom = Geometry.kagome(*args)
        lat, Lx, Ly, per, bx, by = 1, args[0], args[1], 1, args[2], args[2]
    n = geom.n_sites
    t = syn.gaussian_peps(n, 2, 1, seed=1)
    bb = BlockBP(geom, t, chi=4)
    for b in geom.blocks:
        for face in range(4):
            if b.faces[face].nbr is None:
                continue
            trace = []
            bb.update_message(b.id, face, trace=trace) if bb.msgs else None
            if not bb.msgs:
                bb.init_messages(syn.initial_edge_matrices(n, 1, seed=2))
                bb.update_message(b.id, face, trace=trace)
            got = P.bbp_plan_debug(lat, Lx, Ly, per, bx, by, b.id, face)
            want = []
            for rec in trace:
                ident = rec[-1]
                if ident[0] == "site":
                    want.append((0, ident[1], rec[2], rec[3]))
                else:
                    want.append((1, ident[1] * 1024 + ident[2], rec[2], rec[3]))
            assert [tuple(int(x) for x in row) for row in got] == want


def test_partition_rejects_bad_tiling(L):
    with pytest.raises(P.BBPError) as ei:
        P.bbp_plan_debug(0, 6, 6, 0, 4, 3, 0, 2)
    assert ei.value.status == 4
    with pytest.raises(P.BBPError):
        P.bbp_plan_debug(1, 6, 2, 1, 2, 1, 0, 2)      # Kagome blocks must be L x L


def test_null_arguments_return_errors(L):
    assert L.bbp_partition_blocks(None, 3, 3) == 1
    assert L.bbp_iterate(None, 1e-8, 1, None, None) == 1
    assert P.bbp_footprint_bytes(1, 36, 4, 32, 2, 2) > 0


CORES = [
    ("square", (6, 6, 3, 3), 0, [4]),
    ("square", (6, 6, 3, 3), 3, [3, 4]),
    ("square", (6, 6, 3, 3), 0, [1, 4, 5]),
    ("square", (4, 4, 2, 2), 0, [0, 1, 2, 3]),
    ("kagome", (6, 2, 2), 0, "cell"),
    ("kagome", (9, 3, 3), 1, "cell"),
    ("kagome", (9, 3, 3), 0, ("cell", 4)),
    ("kagome", (12, 4, 4), 0, ("cell", 7)),
    ("kagome", (12, 4, 4), 2, ("cell", 12)),
    ("kagome", (6, 2, 2), 0, ("mode", 2)),
    ("kagome", (9, 3, 3), 1, ("mode", 0)),
    ("square", (8, 8, 4, 4), 0, [5, 6]),
    ("square", (8, 8, 4, 4), 3, [9, 10, 13]),
]


def _steps(trace):
    out = []
    for rec in trace:
        ident = rec[-1]
        out.append((0, ident[1], rec[2], rec[3]) if ident[0] == "site" else (1, ident[1] * 1024 + ident[2], rec[2], rec[3]))
    return out


@pytest.mark.parametrize("kind,args,block,core", CORES)
def test_core_plan_matches_oracle_bubbles(L, kind, args, block, core):
    """The host plan of a core extraction (bbp_core_plan_debug) against the
    oracle's two bubbles and zipper (Sec. 2.3): same swallow order and legs
    per step in both bubbles, same boundary lengths, same shared end runs,
    and the same core leg under every pMPS tensor."""
    from oracle import core as C
    if kind == "square":
        geom = Geometry.square(*args)
        lat, Lx, Ly, per, bx, by = 0, args[0], args[1], 0, args[2], args[3]
    else:
        geom = Geometry.kagome(*args)
        lat, Lx, Ly, per, bx, by = 1, args[0], args[1], 1, args[2], args[2]
    n = geom.n_sites
    bb = BlockBP(geom, syn.gaussian_peps(n, 2, 1, seed=1), chi=4)
    bb.init_messages(syn.initial_edge_matrices(n, 1, seed=2))
    b = geom.blocks[block]
    if core == "cell":    # the up-triangle of the block's second unit cell
        i, j = b.sites[2][1:]
        core = [b.sites.index((t, i, j)) for t in range(3)]
    elif isinstance(core, tuple) and core[0] == "mode":   # the first mode through this vertex
        core = next(m for (t, i, j) in b.sites
                    for m in [C.kagome_mode(geom, block, (i, j), core[1])] if m is not None)
    elif isinstance(core, tuple):   # the k-th complete up-triangle of the block
        cells = sorted({(i, j) for (t, i, j) in b.sites if all((u, i, j) in b.sites for u in range(3))})
        i, j = cells[core[1]]
        core = [b.sites.index((t, i, j)) for t in range(3)]
    keys = [(0, q) for q in core]
    traces = []
    region, (B, LB, _), (Tt, LT, _) = C.bubbles(bb, [(b.X, b.Y)], set(keys), traces=traces)
    ring = C.zipper(B, LB, Tt, LT)
    a = 0
    while LB[a] in set(LT):
        a += 1
    c = 0
    while LB[len(LB) - 1 - c] in set(LT):
        c += 1
    sites = {(rs.inst, rs.local): rs for rs in region.sites}
    want_legs = []
    for _, lab in ring:
        want_legs.append(next((k, sites[key].labels.index(lab)) for k, key in enumerate(keys)
                              if lab in sites[key].labels))
    got_b, got_t, (nb, mt, ga, gc, Lr), legs = P.bbp_core_plan_debug(lat, Lx, Ly, per, bx, by, block,
                                                                     [b.gids[q] for q in core])
    assert [tuple(int(x) for x in r) for r in got_b] == _steps(traces[0])
    assert [tuple(int(x) for x in r) for r in got_t] == _steps(traces[1])
    assert (nb, mt, ga, gc, Lr) == (len(LB), len(LT), a, c, len(ring))
    assert legs == want_legs
