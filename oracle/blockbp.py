"""The BlockBP iteration and local observables (test infrastructure only).

Sec. 2.2, Eq. of the BlockBP update: the message a -> b at iteration l is the
contraction of block a with every incoming message of iteration l-1 except
the one from b, compressed to an MPS (boundary-MPS, bond chi).  Alg. 1:
all messages of an iteration are computed from the previous iteration's
messages (synchronous update); an outgoing message becomes the incoming
message of the receiving face (for a block that neighbours itself through a
periodic face, the opposite face of the same block).  Iterate until the
largest message change is at most the threshold (Eq. of the BP convergence
criterion, taken over all messages).

Readings (the thesis leaves these open):
* A: a message is normalised to unit norm <M|M> = 1 as a vector over its
  fused legs, and its global phase is fixed so that its contraction with the
  ket-bra identity <I|M> is real and positive; the change of a message is the
  gauge-invariant distance ||M_new - M_old||, evaluated as the norm of the
  direct-sum MPS (new, -old) (see message_distance).
* B: initial messages are bond-1 MPS built from per-leg D x D positive
  semi-definite matrices supplied as input (see ``synthetic``).
* F: log Z_BP = sum_a log Z_a - sum_{pairs (a,b)} log <M_a->b, M_b->a>,
  with Z_a block a contracted with all its incoming messages.
* Observables: <O> = Z(O) / Z(I), Z from a sweep to the top face followed by
  the plain contraction with the incoming top messages; a bond whose sites
  lie in two blocks is evaluated on the union of the two blocks.
"""
from __future__ import annotations

import math

import numpy as np

from . import learning, tn
from .geometry import TOP, Geometry, DIR_VEC
from .region import block_region, build_region


def normalise_message(mps: list, dims: list):
    """Unit norm and the phase of <I|M> removed (reading A)."""
    mps = [np.array(a) for a in mps]
    nrm2 = tn.mps_overlap(mps, mps).real
    if nrm2 <= 0.0:
        return mps
    mps[0] = mps[0] / math.sqrt(nrm2)
    tr = tn.mps_identity_overlap(mps, dims)
    if abs(tr) > 0.0:
        mps[0] = mps[0] * (abs(tr) / tr)
    return mps


def message_distance(old: list, new: list) -> float:
    """||M_new - M_old|| (reading A).  Computed as the norm of the direct-sum
    MPS of (new, -old) reduced by a left-to-right QR sweep: orthogonal
    reduction keeps the absolute error at rounding level, whereas
    sqrt(2 - 2 Re<old|new>) cannot resolve distances below ~1e-8."""
    k = len(new)
    R = None
    for q in range(k):
        a, b = new[q], old[q]
        la, p, ra = a.shape
        lb, _, rb = b.shape
        if k == 1:
            Dq = (a - b).reshape(1, p, 1)
        elif q == 0:
            Dq = np.concatenate([a, -b], axis=2)
        elif q == k - 1:
            Dq = np.concatenate([a, b], axis=0)
        else:
            Dq = np.zeros((la + lb, p, ra + rb), dtype=np.complex128)
            Dq[:la, :, :ra] = a
            Dq[la:, :, ra:] = b
        if R is not None:
            Dq = np.tensordot(R, Dq, axes=(1, 0))
        l, p, r = Dq.shape
        _, R = np.linalg.qr(Dq.reshape(l * p, r))
    return float(np.linalg.norm(R))


class BlockBP:
    def __init__(self, geom: Geometry, tensors: np.ndarray, chi: int, alpha: float = 1.0,
                 hermitise: bool = False):
        """alpha: learning step (1 = plain replacement); hermitise: replace
        each new message by its Hermitian part (see oracle.learning)."""
        if not 0.0 <= alpha <= 1.0:
            raise ValueError("alpha must lie in [0, 1]")
        self.geom = geom
        self.chi = chi
        self.alpha = alpha
        self.hermitise = hermitise
        self.t = np.asarray(tensors, dtype=np.complex128)
        if self.t.shape[0] != geom.n_sites:
            raise ValueError("one tensor per site expected")
        self.d = self.t.shape[1]
        self.D = self.t.shape[2]
        # site tensors with open legs restricted to index 0 (bond dimension 1)
        self.tc = {}
        for b in geom.blocks:
            for loc, (t_, i, j) in enumerate(b.sites):
                g = b.gids[loc]
                if g in self.tc:
                    continue
                sl = [slice(None)]
                for k in range(4):
                    t2, i2, j2, _ = geom.lattice.neighbour(t_, i, j, k)
                    open_leg = geom.lattice.site_id(t2, i2, j2) is None
                    sl.append(slice(0, 1) if open_leg else slice(None))
                self.tc[g] = self.t[g][tuple(sl)]
        self.T = {g: tn.fuse(tt) for g, tt in self.tc.items()}
        self.msgs = {}
        self.iterations = 0
        self.last_error = math.inf

    # ------------------------------------------------------------ messages --
    def face_dims(self, bid: int, d: int):
        f = self.geom.blocks[bid].faces[d]
        return [1 if e.gid is None else self.D for e in f.edges]

    def init_messages(self, edge_mats: np.ndarray):
        """Bond-1 messages: leg j of the message into (block, face) carries the
        matrix edge_mats[receiving site][its slot] (reading B)."""
        for b in self.geom.blocks:
            for d in range(4):
                f = b.faces[d]
                if f.nbr is None:
                    continue
                mps = []
                for e in f.edges:
                    m = np.asarray(edge_mats[b.gids[e.site]][e.slot], dtype=np.complex128)
                    mps.append(m.reshape(1, -1, 1))
                self.msgs[(b.id, d)] = normalise_message(mps, self.face_dims(b.id, d))

    def incoming(self, bid: int, d: int):
        if (bid, d) in self.msgs:
            return self.msgs[(bid, d)]
        f = self.geom.blocks[bid].faces[d]
        return [np.ones((1, 1, 1), dtype=np.complex128) for _ in f.edges]

    def region_msgs(self, region):
        return {(n, d): self.incoming(region.ids[n], d)
                for d in range(4) for (n, _) in region.side_faces[d]}

    def region_T(self, region, ops=None):
        """Fused tensors of a region; ops maps (instance, local site) -> d x d."""
        ops = ops or {}
        out = {}
        for rs in region.sites:
            key = (rs.inst, rs.local)
            if key in ops:
                out[key] = tn.fuse(self.tc[rs.gid], ops[key])
            else:
                out[key] = self.T[rs.gid]
        return out

    def update_message(self, bid: int, d: int, trace=None):
        """One BlockBP message update: block bid sends through its face d."""
        region = block_region(self.geom, bid)
        msgs = {(0, dd): self.incoming(bid, dd) for dd in range(4)}
        mps, _ = tn.sweep(region, d, self.region_T(region), msgs, self.chi, trace=trace)
        return normalise_message(mps, self.face_dims(bid, d))

    def step(self):
        """One synchronous iteration (Alg. 1); returns the largest change."""
        new = {}
        for (bid, d, recv) in self.geom.updates():
            m = self.update_message(bid, d)
            dims = self.face_dims(*recv)
            if self.hermitise:
                m = normalise_message(learning.hermitise(m, dims, self.chi), dims)
            if self.alpha != 1.0:
                m = normalise_message(learning.learned(m, self.msgs[recv], self.alpha, self.chi), dims)
            new[recv] = m
        err = 0.0
        for key, m in new.items():
            err = max(err, message_distance(self.msgs[key], m))
        self.msgs.update(new)
        self.iterations += 1
        self.last_error = err
        return err

    def run(self, tol: float, max_iter: int):
        err = math.inf
        for _ in range(max_iter):
            err = self.step()
            if err <= tol:
                break
        return self.iterations, err

    # --------------------------------------------------------- observables --
    def contract(self, coords, ops=None):
        """(logscale, value): Z of a region with operators inserted at sites."""
        region = build_region(self.geom, coords)
        msgs = self.region_msgs(region)
        mps, logscale = tn.sweep(region, TOP, self.region_T(region, ops), msgs, self.chi)
        top = []
        for (n, dd) in region.side_faces[TOP]:
            top.extend(msgs[(n, dd)])
        return logscale, tn.mps_overlap(mps, top, conj=False)

    def home(self, g: int):
        """(block, local index) of a global site."""
        for b in self.geom.blocks:
            if g in b.gids:
                return b, b.gids.index(g)
        raise ValueError("site not found")

    def expect(self, ops: dict, coords):
        """<prod O> with ops keyed by (instance, local site) of the region ``coords``."""
        l0, z0 = self.contract(coords)
        l1, z1 = self.contract(coords, ops)
        return z1 / z0 * math.exp(l1 - l0)

    def bond_region(self, g1: int, k1: int):
        """Region and (instance, local) keys of both ends of the bond leaving
        site g1 through slot k1: the block of g1, or the union with the block
        holding the neighbour image (reading E)."""
        geom = self.geom
        b, loc = self.home(g1)
        t_, i, j = b.sites[loc]
        t2, i2, j2, _ = geom.lattice.neighbour(t_, i, j, k1)
        X2, Y2 = geom.part.block_of(t2, i2, j2)
        if (X2, Y2) == (b.X, b.Y):
            coords = [(b.X, b.Y)]
            return coords, (0, loc), (0, b.sites.index((t2, i2, j2)))
        coords = [(b.X, b.Y), (X2, Y2)]
        b2 = geom.blocks[geom.part.block_id(X2, Y2)]
        tx, ty = (X2 - b2.X) * geom.part.bx, (Y2 - b2.Y) * geom.part.by
        return coords, (0, loc), (1, b2.sites.index((t2, i2 - tx, j2 - ty)))

    def bond_expect(self, g1, k1, O1, O2):
        coords, key1, key2 = self.bond_region(g1, k1)
        return self.expect({key1: O1, key2: O2}, coords)

    def site_expect(self, g: int, O):
        b, loc = self.home(g)
        return self.expect({(0, loc): O}, [(b.X, b.Y)])

    def sz(self, g: int) -> complex:
        return self.site_expect(g, np.diag([0.5, -0.5]).astype(np.complex128))

    def heisenberg_bond(self, g1, k1) -> complex:
        sx = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
        sy = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
        sz = np.diag([0.5, -0.5]).astype(np.complex128)
        return sum(self.bond_expect(g1, k1, s, s) for s in (sx, sy, sz))

    def energy_per_site(self):
        bonds = self.geom.bonds()
        e = sum(self.heisenberg_bond(g1, k1) for (g1, k1, _, _) in bonds)
        return e / self.geom.n_sites

    def rdm(self, keys: list, coords):
        """Reduced density matrix of sites given as (instance, local) keys of the
        region ``coords``, from d^(2n) insertions of the basis operators
        |s><s'| (trace-normalised)."""
        d = self.d
        n = len(keys)
        l0, z0 = self.contract(coords)
        dim = d ** n
        rho = np.zeros((dim, dim), dtype=np.complex128)
        for a in range(dim):
            for bb in range(dim):
                ia = np.unravel_index(a, [d] * n)
                ib = np.unravel_index(bb, [d] * n)
                ops = {}
                for q, key in enumerate(keys):
                    E = np.zeros((d, d), dtype=np.complex128)
                    # <psi| (|ib><ia|) |psi> = rho[ia, ib]
                    E[ib[q], ia[q]] = 1.0
                    ops[key] = E
                l1, z1 = self.contract(coords, ops)
                rho[a, bb] = z1 / z0 * math.exp(l1 - l0)
        return rho / np.trace(rho)

    def log_norm(self) -> float:
        """Bethe-form log Z_BP (reading F), real part."""
        total = 0.0 + 0.0j
        for b in self.geom.blocks:
            l, z = self.contract([(b.X, b.Y)])
            total += l + np.log(complex(z))
        seen = set()
        for (bid, d, recv) in self.geom.updates():
            pair = frozenset(((bid, d), recv))
            if pair in seen:
                continue
            seen.add(pair)
            m_in = self.msgs[(bid, d)]        # message into bid on face d
            m_out = self.msgs[recv]           # message into recv, sent by bid through d
            total -= np.log(complex(tn.mps_overlap(m_in, m_out, conj=False)))
        return float(total.real)
