"""Site-level belief propagation (test infrastructure only).

Eq. of BP (Sec. 2.1): m_{a->b} = Tr(T_a prod_{c in N_a \\ b} m_{c->a}), the
double-layer tensor of site a contracted with all its incoming D x D message
matrices except the one from b.  BlockBP with 1 x 1 blocks must reduce to it;
this independent restatement with einsum serves as that pin.  Messages are
normalised and phase-fixed as in ``blockbp`` (reading A).
"""
from __future__ import annotations

import math

import numpy as np

from . import tn
from .geometry import Lattice

_LETTERS = "abcd"


def _normalise(v: np.ndarray, D: int) -> np.ndarray:
    v = v / np.linalg.norm(v)
    tr = sum(v[k * D + k] for k in range(D))
    if abs(tr) > 0.0:
        v = v * (abs(tr) / tr)
    return v


class SiteBP:
    def __init__(self, lat: Lattice, tensors: np.ndarray):
        self.lat = lat
        self.D = tensors.shape[2]
        self.T = {}
        self.nb = {}
        for j in range(lat.Ly):
            for i in range(lat.Lx):
                for t in range(lat.ntypes):
                    g = lat.site_id(t, i, j)
                    row = []
                    sl = [slice(None)]
                    for k in range(4):
                        t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
                        g2 = lat.site_id(t2, i2, j2)
                        row.append(None if g2 is None else (g2, k2))
                        sl.append(slice(None) if g2 is not None else slice(0, 1))
                    self.nb[g] = row
                    self.T[g] = tn.fuse(tensors[g][tuple(sl)])
        self.m = {}   # (g, k) -> message INTO site g on its slot k

    def init(self, edge_mats: np.ndarray):
        for g, row in self.nb.items():
            for k, e in enumerate(row):
                if e is not None:
                    self.m[(g, k)] = _normalise(np.asarray(edge_mats[g][k]).reshape(-1), self.D)

    def outgoing(self, g: int, k_out: int) -> np.ndarray:
        T = self.T[g]
        ops = [T]
        subs = [_LETTERS]
        for k in range(4):
            if k == k_out:
                continue
            if self.nb[g][k] is None:
                v = np.ones(1, dtype=np.complex128)
            else:
                v = self.m[(g, k)]
            ops.append(v)
            subs.append(_LETTERS[k])
        expr = ",".join(subs) + "->" + _LETTERS[k_out]
        return np.einsum(expr, *ops)

    def step(self):
        new = {}
        for g, row in self.nb.items():
            for k, e in enumerate(row):
                if e is None:
                    continue
                g2, k2 = e
                new[(g2, k2)] = _normalise(self.outgoing(g, k), self.D)
        err = 0.0
        for key, v in new.items():
            ov = np.vdot(self.m[key], v).real
            err = max(err, math.sqrt(max(0.0, 2.0 - 2.0 * ov)))
        self.m.update(new)
        return err
