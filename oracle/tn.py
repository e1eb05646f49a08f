"""Tensor-network primitives and the boundary-MPS sweep (test infrastructure only).

* ``fuse``: the double-layer (ket-bra) tensor of Sec. 1.2 / Sec. 2.1,
  T[(u u'), (r r'), ...] = sum_s t[s, u, r, ...] conj(t[s, u', r', ...]),
  a fused leg index being ket * D + bra.  With an operator O inserted:
  T_O = sum_{s, s'} O[s, s'] t[s', ket legs] conj(t[s, bra legs]), so that
  the full contraction gives <psi| O |psi>.
* ``sweep``: the boundary-MPS ("bubblecon") contraction of Sec. 1.1.3 --
  the bubble swallows one tensor at a time; whenever the swallowed tensor
  emits more than one leg, SVDs split the merged tensor back into MPS tensors,
  keeping at most chi singular values (truncation bond dimension chi).  The
  MPS is kept in canonical form (Sec. 2.3.3) with its orthogonality centre
  moved onto the swallowed segment, so each SVD truncates the full state
  optimally at that cut.

Readings (the thesis gives the order only in figures):
* order: nodes sorted by (depth, lateral) in skew coordinates, depth along
  the direction from the start face to the out face;
* legs of the boundary MPS keep the planar order of the boundary; a node's
  out-legs replace its in-legs in reverse counter-clockwise order;
* each split keeps exactly min(chi, rows, cols) singular triplets;
* after each swallow the centre tensor is divided by its Frobenius norm and
  the log of that norm is accumulated (the mantissa/exponent device of
  Sec. 2.3.3, as a natural-log scale).
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import BOTTOM, LEFT, RIGHT, TOP
from .region import Region


# ---------------------------------------------------------------- fusion ----

def fuse(t: np.ndarray, op: np.ndarray | None = None) -> np.ndarray:
    """Double-layer tensor of one site; t has shape (d, D0, D1, D2, D3)."""
    d = t.shape[0]
    dims = t.shape[1:]
    if op is None:
        op = np.eye(d, dtype=np.complex128)
    # T[k0,b0,k1,b1,...] = sum_{s,s'} O[s,s'] t[s',k...] conj(t[s,b...])
    ket = np.tensordot(op, t, axes=(1, 0))            # [s, k0..k3]
    T = np.einsum("sabcd,sefgh->aebfcgdh", ket, np.conj(t))
    return T.reshape([x * x for x in dims])


# ------------------------------------------------------------ MPS helpers ---

def qr_right(A: np.ndarray, B: np.ndarray):
    """Move the orthogonality centre from A to its right neighbour B."""
    l, p, r = A.shape
    Q, R = np.linalg.qr(A.reshape(l * p, r))
    return Q.reshape(l, p, -1), np.tensordot(R, B, axes=(1, 0))


def lq_left(A: np.ndarray, B: np.ndarray):
    """Move the orthogonality centre from B to its left neighbour A."""
    l, p, r = B.shape
    Q, R = np.linalg.qr(B.reshape(l, p * r).conj().T)
    return np.tensordot(A, R.conj().T, axes=(2, 0)), Q.conj().T.reshape(-1, p, r)


def svd_split(R: np.ndarray, chi: int):
    """Split R[l, q1, rest..., r] at (l q1 | rest r) keeping min(chi, rows, cols)."""
    sh = R.shape
    M = R.reshape(sh[0] * sh[1], -1)
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = min(chi, M.shape[0], M.shape[1])
    A1 = U[:, :k].reshape(sh[0], sh[1], k)
    rem = (s[:k, None] * Vh[:k]).reshape((k,) + sh[2:])
    return A1, rem


def mps_overlap(A: list, B: list, conj: bool = True) -> complex:
    """<A|B> (conj=True) or the plain contraction sum A B (conj=False)."""
    E = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(A, B):
        a2 = np.conj(a) if conj else a
        E = np.einsum("xy,xpz,ypw->zw", E, a2, b)
    return complex(E[0, 0])


def mps_identity_overlap(A: list, dims: list) -> complex:
    """<I|A>: contraction of every fused leg with the ket-bra identity."""
    E = np.ones((1,), dtype=np.complex128)
    for a, D in zip(A, dims):
        idx = [k * D + k for k in range(D)]
        E = E @ a[:, idx, :].sum(axis=1)
    return complex(E[0])


def mps_dense(A: list) -> np.ndarray:
    v = np.ones((1, 1), dtype=np.complex128)
    for a in A:
        v = np.tensordot(v, a, axes=(1, 0)).reshape(-1, a.shape[2])
    return v[:, 0]


# ----------------------------------------------------------------- sweep ----

_TANGENT = {BOTTOM: (1.0, 0.0), TOP: (1.0, 0.0), LEFT: (0.0, 1.0), RIGHT: (0.0, 1.0)}


def sweep_key(out_dir: int, p4):
    u, v = p4
    if out_dir == TOP:
        return (v, u)
    if out_dir == BOTTOM:
        return (-v, -u)
    if out_dir == RIGHT:
        return (u, -v)
    return (-u, v)


def _angle(lat, a4, b4) -> float:
    ax, ay = lat.real(a4)
    bx, by = lat.real(b4)
    return math.atan2(by - ay, bx - ax) % (2.0 * math.pi)


class SweepError(RuntimeError):
    pass


def sweep(region: Region, out_dir: int, T: dict, msgs: dict, chi: int, trace: list | None = None,
          skip=None, stop=None, raw: bool = False):
    """Contract a region with the incoming messages of all sides but ``out_dir``.

    T[(inst, local)]   fused site tensor, legs in slot order (dims D^2, or 1 open)
    msgs[(inst, dir)]  incoming MPS on that face, canonical order, tensors (l, p, r)
    Returns (mps, logscale): the MPS over the out side's edges in canonical
    order, and the natural log of the scale factored out along the way.

    A bubble that must leave a core unswallowed (Sec. 2.3, "Core"): ``skip``
    holds the (inst, local) keys of sites that are never swallowed (their
    legs stay open on the boundary), ``stop`` a sweep key at which the bubble
    halts (nodes whose key is >= stop are left), and ``raw`` returns the
    boundary as it stands: (tensors incl. the two end-bond tensors, their leg
    labels in boundary order, logscale).
    """
    lat = region.geom.lattice
    start = (out_dir + 2) % 4
    lo, hi = (out_dir + 1) % 4, (out_dir + 3) % 4
    side_forward = out_dir in (TOP, RIGHT)       # side chains swallowed in canonical order
    chain_forward = out_dir in (TOP, LEFT)        # start/out chains already in lateral order

    def chain_tensors(d):
        out = []
        for (inst, dd) in region.side_faces[d]:
            out.extend(msgs[(inst, dd)])
        return out

    # nodes: (key, kind, payload)
    nodes = []
    node_ident = {}
    for rs in region.sites:
        if skip and (rs.inst, rs.local) in skip:
            continue
        legs = []
        for k in range(4):
            legs.append((rs.labels[k], _angle(lat, rs.pos4, rs.nbr_pos4[k])))
        nodes.append((sweep_key(out_dir, rs.pos4), "site", (rs, legs)))
    for d in (lo, hi):
        edges = region.sides[d]
        tens = chain_tensors(d)
        K = len(edges)
        tx, ty = _TANGENT[d]
        for m, e in enumerate(edges):
            mx, my = lat.real(e.mid4)
            if m > 0:
                px, py = lat.real(edges[m - 1].mid4)
                a_prev = math.atan2(py - my, px - mx) % (2 * math.pi)
            else:
                a_prev = math.atan2(-ty, -tx) % (2 * math.pi)
            if m < K - 1:
                nx, ny = lat.real(edges[m + 1].mid4)
                a_next = math.atan2(ny - my, nx - mx) % (2 * math.pi)
            else:
                a_next = math.atan2(ty, tx) % (2 * math.pi)
            a_phys = _angle(lat, e.mid4, e.inner4)
            legs = [(("b", d, m), a_prev), (e.label, a_phys), (("b", d, m + 1), a_next)]
            node_ident[id(legs)] = (e.face[1], e.index)
            nodes.append((sweep_key(out_dir, e.mid4), "msg", (tens[m], legs)))
    nodes.sort(key=lambda z: z[0])

    def end_label(d, at_start):
        K = len(region.sides[d])
        first = ("b", d, 0)
        last = ("b", d, K)
        if side_forward:
            return first if at_start else last
        return last if at_start else first

    st = chain_tensors(start)
    st_labels = [e.label for e in region.sides[start]]
    if not chain_forward:
        st = [a.transpose(2, 1, 0) for a in reversed(st)]
        st_labels = list(reversed(st_labels))
    one = np.ones((1, 1, 1), dtype=np.complex128)
    A = [one] + [np.array(a, dtype=np.complex128) for a in st] + [one]
    labels = [end_label(lo, True)] + st_labels + [end_label(hi, True)]

    # canonical form: centre at position 0
    for p in range(len(A) - 1, 0, -1):
        A[p - 1], A[p] = lq_left(A[p - 1], A[p])
    c = 0
    logscale = 0.0

    def normalise():
        nonlocal logscale
        n = np.linalg.norm(A[c])
        if n > 0.0:
            A[c] = A[c] / n
            logscale += math.log(n)
        else:
            logscale = -math.inf

    normalise()

    for key, kind, payload in nodes:
        if stop is not None and key >= stop:
            break
        if kind == "site":
            rs, legs = payload
            X = T[(rs.inst, rs.local)]
        else:
            X, legs = payload
        lab = [l for l, _ in legs]
        pos = {l: labels.index(l) for l in lab if l in labels}
        if not pos:
            raise SweepError(f"node {key} has no leg on the boundary")
        ps = sorted(pos.values())
        i, j = ps[0], ps[-1]
        if j - i + 1 != len(ps):
            raise SweepError(f"node {key}: in-legs not contiguous")
        in_order = [labels[p] for p in range(i, j + 1)]
        ccw = sorted(range(len(legs)), key=lambda q: legs[q][1])
        n_in = len(in_order)
        out_ccw = None
        for s0 in range(len(ccw)):
            rot = ccw[s0:] + ccw[:s0]
            if [lab[q] for q in rot[:n_in]] == in_order:
                out_ccw = rot[n_in:]
                break
        if out_ccw is None:
            raise SweepError(f"node {key}: in-legs not in planar order")
        in_idx = [lab.index(l) for l in in_order]
        out_idx = list(reversed(out_ccw))

        # move the orthogonality centre into [i, j]
        while c < i:
            A[c], A[c + 1] = qr_right(A[c], A[c + 1])
            c += 1
        while c > j:
            A[c - 1], A[c] = lq_left(A[c - 1], A[c])
            c -= 1
        # merge the in-segment: S[l, p_i .. p_j, r]
        S = A[i]
        for p in range(i + 1, j + 1):
            S = np.tensordot(S, A[p], axes=(S.ndim - 1, 0))
        Xp = np.transpose(X, in_idx + out_idx)
        nin = len(in_idx)
        R = np.tensordot(S, Xp, axes=(list(range(1, 1 + nin)), list(range(nin))))
        # R[l, r, out...] -> R[l, out..., r]
        R = np.moveaxis(R, 1, R.ndim - 1)
        new_labels = [lab[q] for q in out_idx]
        nout = len(out_idx)
        if trace is not None:
            ident = ("site", rs.gid) if kind == "site" else ("msg",) + node_ident[id(legs)]
            trace.append((key, kind, nin, nout, S.shape[0], S.shape[-1],
                          [X.shape[q] for q in in_idx], [X.shape[q] for q in out_idx], ident))
        if nout == 0:
            if i > 0:
                A[i - 1] = np.tensordot(A[i - 1], R, axes=(2, 0))
                del A[i:j + 1]
                del labels[i:j + 1]
                c = i - 1
            else:
                A[j + 1] = np.tensordot(R, A[j + 1], axes=(1, 0))
                del A[i:j + 1]
                del labels[i:j + 1]
                c = i
        else:
            newA = []
            rem = R
            for _ in range(nout - 1):
                a1, rem = svd_split(rem, chi)
                newA.append(a1)
            newA.append(rem)
            A[i:j + 1] = newA
            labels[i:j + 1] = new_labels
            c = i + nout - 1
        normalise()

    if raw:
        return A, labels, logscale
    # finish: [end(lo), out legs..., end(hi)]
    out_labels = [e.label for e in region.sides[out_dir]]
    exp_lateral = out_labels if chain_forward else list(reversed(out_labels))
    if labels[0] != end_label(lo, False) or labels[-1] != end_label(hi, False) or labels[1:-1] != exp_lateral:
        raise SweepError("final boundary does not match the out side")
    first = A[0].reshape(1, -1)
    A[1] = np.tensordot(first, A[1], axes=(1, 0))
    last = A[-1].reshape(-1, 1)
    A[-2] = np.tensordot(A[-2], last, axes=(2, 0))
    mps = A[1:-1]
    if not chain_forward:
        mps = [a.transpose(2, 1, 0) for a in reversed(mps)]
    return mps, logscale
