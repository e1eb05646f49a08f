"""Hexagonal Kagome blocks and BlockBP on them (test infrastructure only).

Sec. 2.3.1 ("Hexagonal block", "Comparison"), Sec. 2.3 ("Contraction
Order"), App. A.  A hexagonal block of face-length N holds the up-triangles
(unit cells) within hexagonal distance N - 1 of a centre cell: 3N^2 - 3N + 1
cells, N_T = 3(3N^2 - 3N + 1) sites (21 for N = 2, 57 for N = 3).  It has six
faces, named counter-clockwise from the bottom: D, DR, UR, U, UL, DL; every
edge leaving one face enters the opposite face of one neighbouring block.
The block is contracted towards each of its six faces with its own order.
HexCoreEnv extracts a core of the hexagonal block (Sec. 2.3, "Core"), e.g.
the three unit cells around a down-triangle that hold the three "modes".

Readings (the thesis draws the block and two of the six orders only):
* cells (i, j) sit at i a1 + j a2; the hexagonal distance of (i, j) is
  max(|i|, |j|, |i + j|); the blocks tile the lattice along the superlattice
  T1 = (N, N - 1), T2 = (1 - N, 2N - 1) (index 3N^2 - 3N + 1); a periodic
  super-cell Lx x Ly is allowed when (Lx, 0) and (0, Ly) lie on it;
* the face of a crossing edge is the neighbouring block it enters, the six
  neighbours +-T1, +-T2, +-(T2 - T1) taken in angular order from the bottom;
* the sweep towards face f (outward normal at 270 + 60 f degrees) swallows
  nodes by (depth along that normal, lateral along the normal turned by -90
  degrees); the boundary starts as [end bond, the opposite face's message,
  end bond]; the two faces on either side form one side chain each, met in
  order of depth; a face's edges are ordered canonically along the tangent
  of face f mod 3, on both sides of the face;
* sites inside a cell are listed Up (C), Down-Left (A), Down-Right (B), as
  App. A orders them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import tn
from .blockbp import message_distance, normalise_message
from .core import CoreEnv, zipper
from .geometry import Edge, Lattice

FACE_NAMES = ("D", "DR", "UR", "U", "UL", "DL")


def hexdist(i: int, j: int) -> int:
    return max(abs(i), abs(j), abs(i + j))


def _real(p4):
    return ((2 * p4[0] + p4[1]) / 4.0, math.sqrt(3.0) * p4[1] / 4.0)


def _normal(f: int):
    a = math.radians(270.0 + 60.0 * f)
    return (math.cos(a), math.sin(a))


def _key(f: int, p4):
    """(depth, lateral) of a position for the sweep towards face f."""
    x, y = _real(p4)
    nx, ny = _normal(f)
    tx, ty = ny, -nx                     # the normal turned by -90 degrees
    return (round((x * nx + y * ny) * 1e9), round((x * tx + y * ty) * 1e9))


def _canon(f: int, p4) -> float:
    """Canonical position of an edge midpoint along face f (tangent of f mod 3)."""
    x, y = _real(p4)
    nx, ny = _normal(f % 3)
    return x * ny - y * nx


@dataclass
class HexFace:
    block: int
    dir: int
    nbr: int | None = None
    edges: list = field(default_factory=list)


@dataclass
class HexBlock:
    id: int
    centre: tuple              # unwrapped centre cell
    sites: list                # (t, i, j) unwrapped
    gids: list
    pos4: list
    faces: dict                # face -> HexFace


class HexGeometry:
    """Periodic Kagome super-cell cut into hexagonal blocks of face-length N."""

    def __init__(self, N: int, Lx: int, Ly: int):
        if N < 2:
            raise ValueError("face-length N >= 2")
        self.N = N
        r = N - 1
        self.T1, self.T2 = (N, N - 1), (1 - N, 2 * N - 1)
        self.cells_per_block = 3 * N * N - 3 * N + 1
        self.lattice = Lattice("kagome", Lx, Ly, True)
        if not (self._on_superlattice(Lx, 0) and self._on_superlattice(0, Ly)):
            raise ValueError("the super-cell is not a multiple of the hexagonal tiling")
        # centres: the superlattice points inside the super-cell
        centres = set()
        for a in range(-Lx - Ly, Lx + Ly + 1):
            for b in range(-Lx - Ly, Lx + Ly + 1):
                i = a * self.T1[0] + b * self.T2[0]
                j = a * self.T1[1] + b * self.T2[1]
                if 0 <= i < Lx and 0 <= j < Ly:
                    centres.add((i, j))
        self.centres = sorted(centres, key=lambda c: (c[1], c[0]))
        if len(self.centres) * self.cells_per_block != Lx * Ly:
            raise ValueError("the blocks do not tile the super-cell")
        index = {c: n for n, c in enumerate(self.centres)}
        offs = [(di, dj) for dj in range(-r, r + 1) for di in range(-r, r + 1) if hexdist(di, dj) <= r]
        nbrs = [self.T1, self.T2, (self.T2[0] - self.T1[0], self.T2[1] - self.T1[1])]
        nbrs = nbrs + [(-a, -b) for (a, b) in nbrs]

        def angle(v):
            x, y = _real((4 * v[0], 4 * v[1]))
            return (math.degrees(math.atan2(y, x)) - 270.0) % 360.0

        face_of_vec = {}
        for v in nbrs:
            f = int(round(angle(v) / 60.0)) % 6
            if f in face_of_vec.values():
                raise ValueError("neighbour directions do not separate the six faces")
            face_of_vec[v] = f
        self.face_vec = {f: v for v, f in face_of_vec.items()}

        def wrap(i, j):
            return (i % Lx, j % Ly)

        cell_block = {}
        for n, (ci, cj) in enumerate(self.centres):
            for (di, dj) in offs:
                c = wrap(ci + di, cj + dj)
                if c in cell_block:
                    raise ValueError("hexagons overlap")
                cell_block[c] = n
        if len(cell_block) != Lx * Ly:
            raise ValueError("hexagons leave cells uncovered")
        lat = self.lattice
        self.blocks = []
        for n, (ci, cj) in enumerate(self.centres):
            sites = []
            for (di, dj) in sorted(offs, key=lambda o: (o[1], o[0])):
                for t in (2, 0, 1):                       # Up, Down-Left, Down-Right
                    sites.append((t, ci + di, cj + dj))
            idx = {s: q for q, s in enumerate(sites)}
            faces = {f: HexFace(block=n, dir=f) for f in range(6)}
            for q, (t, i, j) in enumerate(sites):
                for k in range(4):
                    t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
                    if (t2, i2, j2) in idx:
                        continue
                    rel = (i2 - ci, j2 - cj)
                    hit = [v for v in nbrs if hexdist(rel[0] - v[0], rel[1] - v[1]) <= r]
                    if len(hit) != 1:
                        raise ValueError("a crossing edge does not enter exactly one neighbouring block")
                    f = face_of_vec[hit[0]]
                    nb = index[wrap(ci + hit[0][0], cj + hit[0][1])]
                    if faces[f].nbr is not None and faces[f].nbr != nb:
                        raise ValueError("a face touches two blocks")
                    faces[f].nbr = nb
                    faces[f].edges.append(Edge(site=q, slot=k, gid=lat.site_id(t2, i2, j2), gslot=k2,
                                               inner4=lat.pos4(t, i, j), outer4=lat.pos4(t2, i2, j2)))
            for f in range(6):
                faces[f].edges.sort(key=lambda e, f=f: _canon(f, e.mid4))
            self.blocks.append(HexBlock(id=n, centre=(ci, cj), sites=sites,
                                        gids=[lat.site_id(*s) for s in sites],
                                        pos4=[lat.pos4(*s) for s in sites], faces=faces))

    def _on_superlattice(self, i: int, j: int) -> bool:
        (a1, b1), (a2, b2) = self.T1, self.T2
        det = a1 * b2 - a2 * b1
        x = i * b2 - a2 * j
        y = a1 * j - b1 * i
        return x % det == 0 and y % det == 0

    @property
    def n_sites(self) -> int:
        return self.lattice.n_sites

    def updates(self):
        return [(b.id, f, (b.faces[f].nbr, (f + 3) % 6)) for b in self.blocks for f in range(6)]

    def home(self, g: int):
        for b in self.blocks:
            if g in b.gids:
                return b, b.gids.index(g)
        raise ValueError("site not found")

    def face_sites(self, b: int, f: int) -> int:
        """Number of distinct block sites with an edge through face f."""
        return len({e.site for e in self.blocks[b].faces[f].edges})


# -------------------------------------------------------------- the sweep --

@dataclass
class _RSite:
    local: int
    gid: int
    pos4: tuple
    labels: list
    nbr_pos4: list


def _region(geom: HexGeometry, b: int):
    blk = geom.blocks[b]
    lat = geom.lattice
    idx = {s: q for q, s in enumerate(blk.sites)}
    sites = []
    for q, (t, i, j) in enumerate(blk.sites):
        labels, nbr = [], []
        for k in range(4):
            t2, i2, j2, k2 = lat.neighbour(t, i, j, k)
            nbr.append(lat.pos4(t2, i2, j2))
            if (t2, i2, j2) in idx:
                labels.append(("i", tuple(sorted(((q, k), (idx[(t2, i2, j2)], k2))))))
            else:
                labels.append(("x", q, k))
        sites.append(_RSite(local=q, gid=blk.gids[q], pos4=blk.pos4[q], labels=labels, nbr_pos4=nbr))
    return sites


def _angle(a4, b4) -> float:
    ax, ay = _real(a4)
    bx, by = _real(b4)
    return math.atan2(by - ay, bx - ax) % (2.0 * math.pi)


def hex_sweep(geom: HexGeometry, b: int, out: int, T: dict, msgs: dict, chi: int, trace: list | None = None,
              skip=None, stop=None, raw: bool = False):
    """Contract block b with its incoming messages on every face but `out`
    towards face `out` (boundary MPS, truncation chi).  T[local] fused site
    tensors (slot order); msgs[f] the incoming MPS on face f, canonical
    order.  Returns (mps over the out face in canonical order, logscale).

    Side-chain bonds carry their physical names (("mb", f, q): the bond
    before canonical tensor q of face f's message; ("mj", f, g): the joint
    of two faces' messages), so that two sweeps of one block name shared
    bonds alike.  skip / stop / raw as in tn.sweep: sites never swallowed,
    the key at which the bubble halts, and the boundary returned as it
    stands (tensors, labels, logscale)."""
    blk = geom.blocks[b]
    sites = _region(geom, b)
    start = (out + 3) % 6
    sides = {"lo": [(out + 2) % 6, (out + 1) % 6], "hi": [(out + 4) % 6, (out + 5) % 6]}
    nodes = []
    for rs in sites:
        if skip and rs.local in skip:
            continue
        legs = [(rs.labels[k], _angle(rs.pos4, rs.nbr_pos4[k])) for k in range(4)]
        nodes.append((_key(out, rs.pos4), "site", (rs, legs)))
    ends = {}
    for side, faces in sides.items():
        chain = []                 # (edge, tensor (prev, p, next), prev label, next label) from the start side
        for f in faces:
            edges = blk.faces[f].edges
            tens = msgs[f]
            order = list(range(len(edges)))
            forward = len(edges) < 2 or _key(out, edges[-1].mid4)[0] > _key(out, edges[0].mid4)[0]
            if not forward:
                order.reverse()
            for q in order:
                a = np.asarray(tens[q])
                pl, nl = (("mb", f, q), ("mb", f, q + 1)) if forward else (("mb", f, q + 1), ("mb", f, q))
                chain.append([edges[q], a if forward else a.transpose(2, 1, 0), pl, nl])
        for m in range(len(chain) - 1):                # the joint of two faces' messages
            if chain[m][3][1] != chain[m + 1][2][1]:
                jl = ("mj",) + tuple(sorted((chain[m][3][1], chain[m + 1][2][1])))
                chain[m][3] = jl
                chain[m + 1][2] = jl
        K = len(chain)
        ends[side] = (chain[0][2], chain[-1][3])
        for m, (e, a, pl, nl) in enumerate(chain):
            mid = e.mid4
            prv = chain[m - 1][0].mid4 if m > 0 else None
            nxt = chain[m + 1][0].mid4 if m < K - 1 else None
            if prv is None:
                prv = (2 * mid[0] - nxt[0], 2 * mid[1] - nxt[1]) if nxt is not None else (mid[0], mid[1] - 1)
            if nxt is None:
                nxt = (2 * mid[0] - prv[0], 2 * mid[1] - prv[1])
            legs = [(pl, _angle(mid, prv)), (("x", e.site, e.slot), _angle(mid, e.inner4)), (nl, _angle(mid, nxt))]
            nodes.append((_key(out, mid), "msg", (a, legs)))
    nodes.sort(key=lambda z: z[0])

    # initial boundary: [lo end, start face in lateral order, hi end]
    st_edges = blk.faces[start].edges
    st = [np.asarray(x) for x in msgs[start]]
    lab = [("x", e.site, e.slot) for e in st_edges]
    lateral_fwd = len(st_edges) < 2 or _key(out, st_edges[-1].mid4)[1] > _key(out, st_edges[0].mid4)[1]
    if not lateral_fwd:
        st = [a.transpose(2, 1, 0) for a in reversed(st)]
        lab = list(reversed(lab))
    one = np.ones((1, 1, 1), dtype=np.complex128)
    A = [one] + [np.array(a, dtype=np.complex128) for a in st] + [one]
    labels = [ends["lo"][0]] + lab + [ends["hi"][0]]
    for p in range(len(A) - 1, 0, -1):
        A[p - 1], A[p] = tn.lq_left(A[p - 1], A[p])
    c = 0
    logscale = 0.0

    def normalise():
        nonlocal logscale
        nrm = np.linalg.norm(A[c])
        if nrm > 0.0:
            A[c] = A[c] / nrm
            logscale += math.log(nrm)
        else:
            logscale = -math.inf

    normalise()
    for key, kind, payload in nodes:
        if stop is not None and key >= stop:
            break
        if kind == "site":
            rs, legs = payload
            X = T[rs.local]
        else:
            X, legs = payload
        lb = [l for l, _ in legs]
        pos = {l: labels.index(l) for l in lb if l in labels}
        if not pos:
            raise tn.SweepError(f"node {key} has no leg on the boundary")
        ps = sorted(pos.values())
        i, j = ps[0], ps[-1]
        if j - i + 1 != len(ps):
            raise tn.SweepError(f"node {key}: in-legs not contiguous")
        in_order = [labels[p] for p in range(i, j + 1)]
        ccw = sorted(range(len(legs)), key=lambda q: legs[q][1])
        n_in = len(in_order)
        out_ccw = None
        for s0 in range(len(ccw)):
            rot = ccw[s0:] + ccw[:s0]
            if [lb[q] for q in rot[:n_in]] == in_order:
                out_ccw = rot[n_in:]
                break
        if out_ccw is None:
            raise tn.SweepError(f"node {key}: in-legs not in planar order")
        in_idx = [lb.index(l) for l in in_order]
        out_idx = list(reversed(out_ccw))
        while c < i:
            A[c], A[c + 1] = tn.qr_right(A[c], A[c + 1])
            c += 1
        while c > j:
            A[c - 1], A[c] = tn.lq_left(A[c - 1], A[c])
            c -= 1
        S = A[i]
        for p in range(i + 1, j + 1):
            S = np.tensordot(S, A[p], axes=(S.ndim - 1, 0))
        Xp = np.transpose(X, in_idx + out_idx)
        nin = len(in_idx)
        R = np.tensordot(S, Xp, axes=(list(range(1, 1 + nin)), list(range(nin))))
        R = np.moveaxis(R, 1, R.ndim - 1)
        new_labels = [lb[q] for q in out_idx]
        nout = len(out_idx)
        if trace is not None:
            trace.append((key, kind, nin, nout))
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
                a1, rem = tn.svd_split(rem, chi)
                newA.append(a1)
            newA.append(rem)
            A[i:j + 1] = newA
            labels[i:j + 1] = new_labels
            c = i + nout - 1
        normalise()
    if raw:
        return A, labels, logscale
    out_edges = blk.faces[out].edges
    want = [("x", e.site, e.slot) for e in out_edges]
    out_fwd = len(out_edges) < 2 or _key(out, out_edges[-1].mid4)[1] > _key(out, out_edges[0].mid4)[1]
    if not out_fwd:
        want = list(reversed(want))
    if labels[0] != ends["lo"][1] or labels[-1] != ends["hi"][1] or labels[1:-1] != want:
        raise tn.SweepError("final boundary does not match the out face")
    first = A[0].reshape(1, -1)
    A[1] = np.tensordot(first, A[1], axes=(1, 0))
    last = A[-1].reshape(-1, 1)
    A[-2] = np.tensordot(A[-2], last, axes=(2, 0))
    mps = A[1:-1]
    if not out_fwd:
        mps = [a.transpose(2, 1, 0) for a in reversed(mps)]
    return mps, logscale


# -------------------------------------------------------- BlockBP on them --

class HexBlockBP:
    """BlockBP (Alg. 1) with hexagonal blocks: every block sends one message
    through each of its six faces, computed from its incoming messages on
    the other five; synchronous updates; readings A and B of the message
    normalisation and initial messages as for the parallelogram blocks."""

    def __init__(self, geom: HexGeometry, tensors: np.ndarray, chi: int):
        self.geom = geom
        self.chi = chi
        self.t = np.asarray(tensors, dtype=np.complex128)
        self.d, self.D = self.t.shape[1], self.t.shape[2]
        self.tc = {g: self.t[g] for g in range(geom.n_sites)}     # (periodic: no open legs)
        self.T = {g: tn.fuse(self.t[g]) for g in range(geom.n_sites)}
        self.msgs = {}

    def face_dims(self, b: int, f: int):
        return [self.D for _ in self.geom.blocks[b].faces[f].edges]

    def init_messages(self, edge_mats: np.ndarray):
        for blk in self.geom.blocks:
            for f in range(6):
                mps = [np.asarray(edge_mats[blk.gids[e.site]][e.slot], dtype=np.complex128).reshape(1, -1, 1)
                       for e in blk.faces[f].edges]
                self.msgs[(blk.id, f)] = normalise_message(mps, self.face_dims(blk.id, f))

    def block_T(self, b: int, ops=None):
        ops = ops or {}
        blk = self.geom.blocks[b]
        return {q: (tn.fuse(self.t[g], ops[q]) if q in ops else self.T[g]) for q, g in enumerate(blk.gids)}

    def update_message(self, b: int, f: int, trace=None):
        msgs = {ff: self.msgs[(b, ff)] for ff in range(6)}
        mps, _ = hex_sweep(self.geom, b, f, self.block_T(b), msgs, self.chi, trace=trace)
        return normalise_message(mps, self.face_dims(b, f))

    def step(self):
        new = {}
        for (b, f, recv) in self.geom.updates():
            new[recv] = self.update_message(b, f)
        err = max(message_distance(self.msgs[k], m) for k, m in new.items())
        self.msgs.update(new)
        return err

    def run(self, tol: float, max_iter: int):
        err = math.inf
        it = 0
        for it in range(1, max_iter + 1):
            err = self.step()
            if err <= tol:
                break
        return it, err

    def contract(self, b: int, ops=None, towards: int = 3):
        """(logscale, Z) of block b with all its incoming messages, swept
        towards face `towards` and closed with the incoming message there."""
        msgs = {ff: self.msgs[(b, ff)] for ff in range(6)}
        mps, ls = hex_sweep(self.geom, b, towards, self.block_T(b, ops), msgs, self.chi)
        return ls, tn.mps_overlap(mps, msgs[towards], conj=False)

    def expect(self, b: int, ops: dict):
        l0, z0 = self.contract(b)
        l1, z1 = self.contract(b, ops)
        return z1 / z0 * math.exp(l1 - l0)


class HexCoreEnv(CoreEnv):
    """The core of a hexagonal block with its pMPS (Sec. 2.3, "Core"): the
    bubbles start from the bottom (D) and top (U) faces, the bottom one
    swallowing every node before the core's last site in the bottom-up
    order, the top one every node after it; the zipper joins them (see
    core.zipper).  Values, RDMs and Edge TNs as for CoreEnv; sites are keyed
    by their local index in the block."""

    def __init__(self, bbp: HexBlockBP, b: int, core_locals):
        self.bbp = bbp
        self.core = list(core_locals)
        geom = bbp.geom
        blk = geom.blocks[b]
        self.sites = {rs.local: rs for rs in _region(geom, b)}
        if not self.core or any(q not in self.sites for q in self.core):
            raise ValueError("core sites must be sites of the block")
        last = max(self.core, key=lambda q: _key(3, blk.pos4[q]))
        p4 = blk.pos4[last]
        T = bbp.block_T(b)
        msgs = {f: bbp.msgs[(b, f)] for f in range(6)}
        skip = set(self.core)
        B, LB, lsB = hex_sweep(geom, b, 3, T, msgs, bbp.chi, skip=skip, stop=_key(3, p4), raw=True)
        Tt, LT, lsT = hex_sweep(geom, b, 0, T, msgs, bbp.chi, skip=skip, stop=_key(0, p4), raw=True)
        self.pmps = zipper(B, LB, Tt, LT)
        self.logscale = lsB + lsT
        self.parts = (B, LB, Tt, LT)
