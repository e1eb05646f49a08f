"""Brute-force exact contraction of small finite lattices (test infrastructure only).

<psi| O |psi> of a finite PEPS is the full contraction of its double-layer
network (Sec. 1.2 / Sec. 2.1) with operators inserted.  Tensors are absorbed
one at a time into a dense boundary tensor, with no truncation at all, so the
result is exact up to rounding.  Used to pin the boundary-MPS sweep, the
tree-of-blocks exactness of BlockBP, and the config-1 comparison.
"""
from __future__ import annotations

import numpy as np

from . import tn
from .geometry import Lattice


def contract_network(items) -> complex:
    """items: list of (array, labels); every label appears on exactly two arrays."""
    B = np.ones((), dtype=np.complex128)
    labels: list = []
    for X, lx in items:
        shared = [l for l in lx if l in labels]
        B = np.tensordot(B, X, axes=([labels.index(l) for l in shared], [lx.index(l) for l in shared]))
        labels = [l for l in labels if l not in shared] + [l for l in lx if l not in shared]
    if labels:
        raise ValueError("dangling labels left")
    return complex(B)


def site_network(lat: Lattice, tensors: np.ndarray, ops: dict | None = None):
    """Fused tensors of a finite lattice with labelled legs, open legs removed."""
    ops = ops or {}
    items = []
    order = []
    for j in reversed(range(lat.Ly)):          # top row first
        for i in range(lat.Lx):
            for t in range(lat.ntypes):
                order.append((t, i, j))
    for (t, i, j) in order:
        g = lat.site_id(t, i, j)
        sl = [slice(None)]
        labels = []
        for k in range(4):
            t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
            g2 = lat.site_id(t2, i2, j2)
            if g2 is None:
                sl.append(slice(0, 1))
                labels.append(None)
            else:
                sl.append(slice(None))
                labels.append(tuple(sorted(((g, k), (g2, k2)))))
        T = tn.fuse(tensors[g][tuple(sl)], ops.get(g))
        keep = [k for k in range(4) if labels[k] is not None]
        T = T.reshape([T.shape[k] for k in keep])
        items.append((T, [labels[k] for k in keep]))
    return items


def norm(lat: Lattice, tensors: np.ndarray) -> complex:
    return contract_network(site_network(lat, tensors))


def expect(lat: Lattice, tensors: np.ndarray, ops: dict) -> complex:
    z0 = contract_network(site_network(lat, tensors))
    z1 = contract_network(site_network(lat, tensors, ops))
    return z1 / z0


def rdm(lat: Lattice, tensors: np.ndarray, gids: list, d: int = 2) -> np.ndarray:
    n = len(gids)
    dim = d ** n
    z0 = contract_network(site_network(lat, tensors))
    rho = np.zeros((dim, dim), dtype=np.complex128)
    for a in range(dim):
        for b in range(dim):
            ia = np.unravel_index(a, [d] * n)
            ib = np.unravel_index(b, [d] * n)
            ops = {}
            for q, g in enumerate(gids):
                E = np.zeros((d, d), dtype=np.complex128)
                E[ib[q], ia[q]] = 1.0
                ops[g] = E
            rho[a, b] = contract_network(site_network(lat, tensors, ops)) / z0
    return rho
