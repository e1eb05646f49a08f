"""Core extraction, the periodic MPS around it, and the Edge TN (test infrastructure only).

Sec. 2.3 ("Core", "Modes", "Edge"): once the messages have converged, a
unit cell is held in the middle of its block and everything else -- the rest
of the block and all its incoming messages -- is contracted into a periodic
MPS (pMPS) around it:

1. two bubblecon sweeps start from opposite faces of the block and approach
   each other; neither swallows the core, so they meet at two front lines
   that touch everywhere except at the core;
2. the two resulting MPSs are joined where they touch, like closing a
   zipper, which leaves one periodic MPS whose open legs are exactly the
   legs of the core;
3. local quantities of the core (one-site and bond expectation values,
   reduced density matrices) are exact contractions of the core's tensors
   with that pMPS; contracting every core site but the two ends of one bond
   gives the Edge TN, the environment of that bond used by the ITE update
   (Sec. 3.2).

Readings (the thesis shows these steps only in figures):
* the bubble from the bottom face swallows, in the bottom-up sweep order,
  every node that comes before the last core site; the bubble from the top
  face swallows, in the top-down order, every node that comes after it; the
  core sites are skipped by both (Sec. 2.3's core is any connected set of
  sites, e.g. one unit cell; the parallelogram block of this engine has four
  faces, so the two bubbles start from its bottom and top faces);
* each bubble truncates to chi exactly as the message update does; the
  zipper itself is exact (no truncation);
* the pMPS is stored as one 3-leg tensor per open core leg, in cyclic order;
  the two zipper matrices are folded into the tensor before them;
* the three "modes" of the hexagonal core are specific to the 6-fold block
  and are not formed here; the Edge TN is taken directly from the core.
"""
from __future__ import annotations

import numpy as np

from . import tn
from .geometry import BOTTOM, TOP
from .region import build_region


class ZipError(RuntimeError):
    pass


def bubbles(bbp, coords, core: set, traces: list | None = None):
    """The two bubbles of step 1 around the core sites ``core`` ((inst, local)
    keys) of the region ``coords``.  Returns (B, LB, lsB), (Tt, LT, lsT): the
    bottom-up and top-down boundary MPSs with their leg labels in boundary
    order and their log scales.  ``traces``, if given, receives the swallow
    records of the two sweeps (see tn.sweep)."""
    region = build_region(bbp.geom, coords)
    keys = {(rs.inst, rs.local): rs for rs in region.sites}
    if not core or any(k not in keys for k in core):
        raise ValueError("core sites must be sites of the region")
    T = bbp.region_T(region)
    msgs = bbp.region_msgs(region)
    last = max(core, key=lambda k: tn.sweep_key(TOP, keys[k].pos4))
    p4 = keys[last].pos4
    tb, tt = ([], []) if traces is not None else (None, None)
    B, LB, lsB = tn.sweep(region, TOP, T, msgs, bbp.chi, trace=tb, skip=core, stop=tn.sweep_key(TOP, p4), raw=True)
    Tt, LT, lsT = tn.sweep(region, BOTTOM, T, msgs, bbp.chi, trace=tt, skip=core, stop=tn.sweep_key(BOTTOM, p4),
                           raw=True)
    if traces is not None:
        traces.extend([tb, tt])
    return region, (B, LB, lsB), (Tt, LT, lsT)


def zipper(B, LB, Tt, LT):
    """Step 2: join the two bubbles where they share legs.

    B runs laterally left to right, Tt right to left, so B's leading shared
    legs meet Tt's trailing ones (front line on the left) and B's trailing
    shared legs meet Tt's leading ones (front line on the right).  Each front
    line is contracted into one matrix, E_L[b, t] and E_R[b, t], b a bond of B
    and t a bond of Tt next to the core.  Returns the pMPS: a list of
    (tensor (l, p, r), physical label) in cyclic order -- B's core legs, then
    Tt's core legs -- with E_R folded into the last tensor of B's part and E_L
    into the last tensor of Tt's part, so that the right bond of the last
    tensor is the left bond of the first."""
    shared = set(LB) & set(LT)
    n, m = len(LB), len(LT)
    a = 0
    while a < n and LB[a] in shared:
        a += 1
    c = 0
    while c < n - a and LB[n - 1 - c] in shared:
        c += 1
    if a == 0 or c == 0:
        raise ZipError("the bubbles do not share both end bonds")
    if LB[:a] != LT[m - a:][::-1] or LB[n - c:] != LT[:c][::-1]:
        raise ZipError("the front lines of the two bubbles do not match")
    core_B = list(range(a, n - c))
    core_T = list(range(c, m - a))
    if any(LB[q] in shared for q in core_B) or any(LT[q] in shared for q in core_T):
        raise ZipError("a shared leg lies between the core legs")
    # left front line: B[0 .. a-1] against Tt[m-1 .. m-a]
    EL = np.ones((1, 1), dtype=np.complex128)
    for q in range(a):
        EL = np.einsum("xy,xpz,wpy->zw", EL, B[q], Tt[m - 1 - q])
    # right front line: B[n-1 .. n-c] against Tt[0 .. c-1]
    ER = np.ones((1, 1), dtype=np.complex128)
    for q in range(c):
        ER = np.einsum("zw,xpz,wpy->xy", ER, B[n - 1 - q], Tt[q])
    # cyclic order: B core part, E_R (B bond -> Tt bond), Tt core part, E_L^T
    items = [("t", B[q], LB[q]) for q in core_B] + [("m", ER, None)]
    items += [("t", Tt[q], LT[q]) for q in core_T] + [("m", EL.T, None)]
    if not any(kind == "t" for kind, _, _ in items):
        raise ZipError("the core has no open legs")
    while items[0][0] != "t":
        items = items[1:] + items[:1]
    pmps = []
    for kind, X, lab in items:
        if kind == "t":
            pmps.append([np.array(X), lab])
        else:
            pmps[-1][0] = np.tensordot(pmps[-1][0], X, axes=(2, 0))
    for q in range(len(pmps)):
        if pmps[q][0].shape[2] != pmps[(q + 1) % len(pmps)][0].shape[0]:
            raise ZipError("pMPS bonds do not close")
    return [(X, lab) for X, lab in pmps]


class CoreEnv:
    """The core of a region together with its pMPS (steps 1 and 2)."""

    def __init__(self, bbp, coords, core_keys):
        self.bbp = bbp
        self.core = list(core_keys)
        region, (B, LB, lsB), (Tt, LT, lsT) = bubbles(bbp, coords, set(self.core))
        self.region = region
        self.sites = {(rs.inst, rs.local): rs for rs in region.sites}
        self.pmps = zipper(B, LB, Tt, LT)
        self.logscale = lsB + lsT
        self.parts = (B, LB, Tt, LT)

    def pmps_items(self):
        L = len(self.pmps)
        return [(X, [("ring", q), lab, ("ring", (q + 1) % L)]) for q, (X, lab) in enumerate(self.pmps)]

    def core_items(self, ops=None, keys=None):
        ops = ops or {}
        out = []
        for k in (keys if keys is not None else self.core):
            rs = self.sites[k]
            X = tn.fuse(self.bbp.tc[rs.gid], ops[k]) if k in ops else self.bbp.T[rs.gid]
            out.append((X, list(rs.labels)))
        return out

    def value(self, ops=None):
        """Step 3: (logscale, Z) of the core with operators ops[(inst, local)]
        inserted, contracted exactly with the pMPS."""
        return self.logscale, complex(contract_open(self.pmps_items() + self.core_items(ops), []))

    def expect(self, ops):
        _, z0 = self.value()
        _, z1 = self.value(ops)
        return z1 / z0

    def rdm(self, keys):
        """Reduced density matrix of core sites (same basis and normalisation as
        BlockBP.rdm): rho[a, b] from insertions of |ib><ia| on every site."""
        d = self.bbp.d
        n = len(keys)
        dim = d ** n
        _, z0 = self.value()
        rho = np.zeros((dim, dim), dtype=np.complex128)
        for a in range(dim):
            for b in range(dim):
                ia = np.unravel_index(a, [d] * n)
                ib = np.unravel_index(b, [d] * n)
                ops = {}
                for q, k in enumerate(keys):
                    E = np.zeros((d, d), dtype=np.complex128)
                    E[ib[q], ia[q]] = 1.0
                    ops[k] = E
                rho[a, b] = self.value(ops)[1] / z0
        return rho / np.trace(rho)

    def edge(self, k1, k2):
        """The Edge TN of the bond between core sites k1 and k2: the pMPS with
        every other core site contracted into it, returned as a dense tensor
        N over the legs of k1 and k2 that do not join them (fused ket-bra
        legs), with those legs' labels in order: (N, labels, slots), where
        slots[q] = (key, slot) names the site leg of labels[q]."""
        rs1, rs2 = self.sites[k1], self.sites[k2]
        joint = set(rs1.labels) & set(rs2.labels)
        if len(joint) != 1:
            raise ValueError("the two sites must share exactly one bond")
        others = [k for k in self.core if k not in (k1, k2)]
        open_legs, slots = [], []
        for k, rs in ((k1, rs1), (k2, rs2)):
            for s, lab in enumerate(rs.labels):
                if lab not in joint:
                    open_legs.append(lab)
                    slots.append((k, s))
        items = self.pmps_items() + self.core_items(keys=others)
        return contract_open(items, open_legs), open_legs, slots


def contract_open(items, open_labels):
    """Dense contraction of labelled arrays, leaving ``open_labels`` (each on
    exactly one array) as the result's axes in that order; every other label
    appears on exactly two arrays.  The arrays are taken one at a time,
    each time the one connected to what is already contracted that leaves
    the smallest intermediate (an order only: the contraction is exact)."""
    pending = list(items)
    Bt = np.ones((), dtype=np.complex128)
    labels: list = []
    while pending:
        best, best_size = 0, None
        for n, (X, lx) in enumerate(pending):
            shared = [l for l in lx if l in labels]
            if labels and not shared:
                continue
            size = 1
            for q, l in enumerate(labels):
                if l not in shared:
                    size *= Bt.shape[q]
            for q, l in enumerate(lx):
                if l not in shared:
                    size *= X.shape[q]
            if best_size is None or size < best_size:
                best, best_size = n, size
        X, lx = pending.pop(best)
        shared = [l for l in lx if l in labels]
        Bt = np.tensordot(Bt, X, axes=([labels.index(l) for l in shared], [lx.index(l) for l in shared]))
        labels = [l for l in labels if l not in shared] + [l for l in lx if l not in shared]
    if sorted(map(repr, labels)) != sorted(map(repr, open_labels)):
        raise ValueError("open labels do not match")
    return np.transpose(Bt, [labels.index(l) for l in open_labels])


def edge_rdm(N, slots, d, D1, D2, t1, t2, s1, s2):
    """Two-site RDM from an Edge TN: N over the fused open legs of sites 1 and 2
    (slots as returned by CoreEnv.edge), t1 / t2 the site tensors (d, legs in
    slot order), s1 / s2 the slots of the joining bond.  rho[(a1 a2), (b1 b2)]
    = <psi| |b1 b2><a1 a2| |psi> / Z, the convention of BlockBP.rdm."""
    ket = np.einsum(two_site_spec(s1, s2), t1, t2)          # [p1, p2, open legs of 1, open legs of 2]
    nopen = ket.ndim - 2
    # fused leg q of N = ket index * Dq + bra index
    dims = ket.shape[2:]
    Nu = N.reshape([x for q in range(nopen) for x in (dims[q], dims[q])])
    kidx = list(range(0, 2 * nopen, 2))
    bidx = list(range(1, 2 * nopen, 2))
    Nkb = np.transpose(Nu, kidx + bidx).reshape(int(np.prod(dims)), int(np.prod(dims)))
    K = ket.reshape(d * d, -1)
    # Z(O) = sum_{s, s'} O[s, s'] M[s', s] with M[s', s] = sum_{k, b} N[k, b] psi[s', k] conj(psi[s, b]);
    # inserting O = |b><a| gives rho[a, b] = M[a, b]
    rho = K @ Nkb @ K.conj().T
    return rho / np.trace(rho)


def two_site_spec(s1: int, s2: int) -> str:
    """einsum spec joining t1 (d, 4 legs) and t2 (d, 4 legs) over slot s1 of t1
    and slot s2 of t2: result [p1, p2, t1's other legs, t2's other legs]."""
    a = ["b", "c", "d", "e"]
    b = ["f", "g", "h", "i"]
    b[s2] = a[s1]
    out = "xy" + "".join(a[q] for q in range(4) if q != s1) + "".join(b[q] for q in range(4) if q != s2)
    return "x" + "".join(a) + ",y" + "".join(b) + "->" + out



# Down-triangle bonds of the Kagome lattice (Sec. 2.3.1): B(R)-A(R + a1),
# C(R)-A(R + a2), B(R)-C(R + a1 - a2); through each vertex of the up-triangle
# of cell R runs one down-triangle: its two other sites as (type, di, dj).
_DOWN_THROUGH = {0: ((1, -1, 0), (2, 0, -1)),      # A(R): B(R - a1), C(R - a2)
                 1: ((0, 1, 0), (2, 1, -1)),       # B(R): A(R + a1), C(R + a1 - a2)
                 2: ((0, 0, 1), (1, -1, 1))}       # C(R): A(R + a2), B(R - a1 + a2)


def kagome_mode(geom, bid: int, cell, vertex: int):
    """A mode (Sec. 2.3, "Modes") of a parallelogram Kagome block: the
    up-triangle A, B, C of unit cell `cell` and the down-triangle through
    its `vertex` (0 A, 1 B, 2 C), five sites holding each of the six bond
    types of the three-site unit cell once.  Returns the local indices
    (up-triangle first), or None when a site lies outside the block."""
    blk = geom.blocks[bid]
    i, j = cell
    sites = [(t, i, j) for t in range(3)]
    for (t, di, dj) in _DOWN_THROUGH[vertex]:
        sites.append((t, i + di, j + dj))
    if any(s not in blk.sites for s in sites):
        return None
    return [blk.sites.index(s) for s in sites]


def bond_type(lat, t: int, k: int):
    """The bond type of leg k of a type-t site: its two (type, slot) ends."""
    t2, _, _, k2 = lat.neighbour(t, 0, 0, k)
    return tuple(sorted(((t, k), (t2, k2))))
