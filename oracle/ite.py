"""Imaginary time evolution with ALS on the BlockBP Edge environment (test infrastructure only).

Ch. 3.  One ITE step on a bond (i, j) (Sec. 3.2, "ITE update step"):
1. evolution: the ket tensors t_i, t_j are contracted with the two-site gate
   exp(-dt h_ij) through their physical legs, giving the exact two-site
   tensor of |psi'>, whose bond between i and j is wider than D;
2. truncation: new tensors t_i, t_j of bond D minimise
   Phi(t_i, t_j) = || |psi> - |psi'> ||^2
                 = <psi|psi> + <psi'|psi'> - <psi|psi'> - <psi'|psi>,
   every scalar taken with the environment N_ij of the bond (the Edge TN of
   Sec. 2.3, from the converged BlockBP messages);
3. ALS: starting from a split of |psi'>, fix t_j and minimise Phi over t_i
   (a linear least-squares problem), then fix t_i and minimise over t_j,
   and repeat until Phi stops decreasing.
Full ITE (Alg. 2): for every time step, for every bond of the block: run
BlockBP, take the bond's Edge TN, update the two tensors by ALS, put them
back; the bonds are visited forwards and then backwards with half steps
(second-order Trotter splitting).  full_ite_unit_cell is the Kagome form of
Sec. 3.3: one unit cell's three tensors repeated over the lattice, the six
bonds of a mode updated, the new tensors copied to every site of their
type (the thesis' random block rotations and mode shuffling are left out).

Readings:
* the start of ALS is the truncated SVD of the evolved two-site tensor
  across the bond (D kept), its singular values split evenly (sqrt) between
  the two sides; the thesis starts from "t_i = t'_i" without saying how the
  wider bond is brought back to D;
* each half-step solves the normal equations M x = c of the quadratic
  Phi with a least-squares routine (M may be singular); the environment
  enters through its Hermitian part;
* als uses the full environment; als_reduced is the thesis' variant (QR of
  each site tensor over its outer legs, the isometric Q moved into the
  environment, ALS on the small R parts), which it reports gives similar
  results at a lower cost;
* after each update both tensors are divided by their largest entry (the
  state is defined up to normalisation; observables are ratios).
"""
from __future__ import annotations

import numpy as np

from .blockbp import BlockBP
from .core import CoreEnv, two_site_spec

SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.diag([0.5, -0.5]).astype(np.complex128)


def heisenberg_h() -> np.ndarray:
    """S_i . S_j as a 4 x 4 matrix over (s_i s_j) (index s_i * 2 + s_j)."""
    return sum(np.kron(S, S) for S in (SX, SY, SZ))


def gate(h: np.ndarray, dt: float) -> np.ndarray:
    """exp(-dt h) of a Hermitian h, through its eigendecomposition."""
    w, V = np.linalg.eigh(h)
    return (V * np.exp(-dt * w)) @ V.conj().T


def evolve(t1, t2, s1, s2, G):
    """Step 1: Theta[p1, p2, open legs of 1, open legs of 2] = sum G[(p1 p2), (q1 q2)]
    t1[q1, ...] t2[q2, ...], the bond joining slot s1 of t1 and slot s2 of t2
    contracted."""
    d = t1.shape[0]
    psi = np.einsum(two_site_spec(s1, s2), t1, t2)
    sh = psi.shape
    out = G @ psi.reshape(d * d, -1)
    return out.reshape(sh)


def _insert(core: np.ndarray, slot: int) -> np.ndarray:
    """[p, other legs (3, slot order), bond] -> [p, 4 legs] with the bond at slot."""
    others = [q for q in range(4) if q != slot]
    order = [None] * 5
    order[0] = 0
    for k, q in enumerate(others):
        order[1 + q] = 1 + k
    order[1 + slot] = 4
    return np.transpose(core, order)


def split(Theta, s1, s2, D):
    """Start of ALS: the truncated SVD of Theta across the bond, D kept."""
    d = Theta.shape[0]
    o1 = Theta.shape[2:5]
    o2 = Theta.shape[5:8]
    M = np.transpose(Theta, (0, 2, 3, 4, 1, 5, 6, 7)).reshape(d * int(np.prod(o1)), d * int(np.prod(o2)))
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = min(D, len(s))
    sq = np.sqrt(s[:k])
    A = (U[:, :k] * sq).reshape((d,) + tuple(o1) + (k,))
    B = (sq[:, None] * Vh[:k]).reshape((k, d) + tuple(o2))
    B = np.moveaxis(B, 0, -1)
    if k < D:                          # keep bond dimension D (zero padding)
        A = np.concatenate([A, np.zeros(A.shape[:-1] + (D - k,), A.dtype)], axis=-1)
        B = np.concatenate([B, np.zeros(B.shape[:-1] + (D - k,), B.dtype)], axis=-1)
    return _insert(A, s1), _insert(B, s2)


def env_matrix(N: np.ndarray, dims1, dims2) -> np.ndarray:
    """The Edge TN (fused ket-bra legs, order: site 1's open legs, site 2's)
    as a matrix N[K, B], K = (ket legs of 1, ket legs of 2), B likewise bra;
    its Hermitian part, so that Phi is real (an exact environment is
    Hermitian; truncation leaves a small anti-Hermitian part)."""
    dims = list(dims1) + list(dims2)
    n = len(dims)
    Nu = N.reshape([x for q in range(n) for x in (dims[q], dims[q])])
    Nkb = np.transpose(Nu, list(range(0, 2 * n, 2)) + list(range(1, 2 * n, 2)))
    size = int(np.prod(dims))
    Nkb = Nkb.reshape(size, size)
    return 0.5 * (Nkb + Nkb.conj().T)


def _two_site(t1, t2, s1, s2):
    psi = np.einsum(two_site_spec(s1, s2), t1, t2)
    d = t1.shape[0]
    return psi.reshape(d * d, -1)


def phi(t1, t2, s1, s2, Nkb, Theta) -> float:
    """Phi = <psi - psi'| N |psi - psi'> (Eq. of the ITE minimisation function)."""
    d = t1.shape[0]
    X = _two_site(t1, t2, s1, s2) - Theta.reshape(d * d, -1)
    return float(np.einsum("pk,kb,pb->", X, Nkb, X.conj()).real)


def _open(t, s):
    """[p, 4 legs] -> [p, other legs flattened, bond]."""
    others = [q for q in range(4) if q != s]
    X = np.transpose(t, [0] + [1 + q for q in others] + [1 + s])
    return X.reshape(X.shape[0], -1, X.shape[-1])


def _close(X, t_like, s):
    """Inverse of _open for a tensor shaped like t_like."""
    others = [q for q in range(4) if q != s]
    shape = [t_like.shape[0]] + [t_like.shape[1 + q] for q in others] + [t_like.shape[1 + s]]
    Y = X.reshape(shape)
    return _insert(Y, s)


def solve_site(x_t, y_t, s1, s2, Nkb, Theta, first: bool):
    """One ALS half-step: returns the site-1 tensor minimising Phi with the
    site-2 tensor fixed (first=True), or the site-2 tensor with site 1 fixed."""
    d = x_t.shape[0]
    x = _open(x_t, s1)                               # [p1, E1, bond]
    y = _open(y_t, s2)                               # [p2, E2, bond]
    E1, E2, Dv = x.shape[1], y.shape[1], x.shape[2]
    N4 = Nkb.reshape(E1, E2, E1, E2)                 # [K1, K2, B1, B2]
    Th4 = Theta.reshape(d, d, E1, E2)                # [p1, p2, K1, K2]
    if first:
        # quadratic part sum conj(x[p1, B1, b']) M[(B1 b'), (K1 b)] x[p1, K1, b]
        M = np.einsum("kKbB,pKc,pBe->bekc", N4, y, y.conj()).reshape(E1 * Dv, E1 * Dv)
        # linear part sum conj(x[p1, B1, b']) c[p1, B1, b'] (and its conjugate)
        c = np.einsum("kKbB,qpkK,pBe->qbe", N4, Th4, y.conj()).reshape(d, E1 * Dv)
        like, slot = x_t, s1
    else:
        M = np.einsum("kKbB,pkc,pbe->BeKc", N4, x, x.conj()).reshape(E2 * Dv, E2 * Dv)
        c = np.einsum("kKbB,pqkK,pbe->qBe", N4, Th4, x.conj()).reshape(d, E2 * Dv)
        like, slot = y_t, s2
    # stationary point of the quadratic form: M v_p = c_p for every physical index p
    V = np.stack([np.linalg.lstsq(M, c[p], rcond=1e-13)[0] for p in range(d)])
    return _close(V, like, slot)


def als(t1, t2, s1, s2, N, dims1, dims2, G, D, max_sweeps: int = 50, tol: float = 1e-13):
    """Steps 1-3 for one bond.  Returns (t1, t2, history of Phi): Phi after
    the SVD start and after every half-step."""
    Theta = evolve(t1, t2, s1, s2, G)
    Nkb = env_matrix(N, dims1, dims2)
    a, b = split(Theta, s1, s2, D)
    hist = [phi(a, b, s1, s2, Nkb, Theta)]
    for _ in range(max_sweeps):
        a = solve_site(a, b, s1, s2, Nkb, Theta, True)
        hist.append(phi(a, b, s1, s2, Nkb, Theta))
        b = solve_site(a, b, s1, s2, Nkb, Theta, False)
        hist.append(phi(a, b, s1, s2, Nkb, Theta))
        if hist[-3] - hist[-1] <= tol * max(abs(hist[0]), 1e-300):
            break
    return a, b, hist


def reduce_site(t, s):
    """The reduced-environment split of one site tensor (Sec. 3.2): a QR over
    its outer legs, t[p, outer, bond] = sum_k Q[outer, k] r[p, k, bond], Q an
    isometry that joins the environment and r (d x k x D) the part ALS
    updates."""
    x = _open(t, s)                                   # [p, E, bond]
    d, E, Db = x.shape
    Q, R = np.linalg.qr(np.transpose(x, (1, 0, 2)).reshape(E, d * Db))
    k = Q.shape[1]
    return Q, np.transpose(R.reshape(k, d, Db), (1, 0, 2))


def reduced_env(N, dims1, dims2, Q1, Q2):
    """The environment seen by the reduced tensors: N with site 1's outer
    legs contracted with Q1 (ket) and conj(Q1) (bra), site 2's with Q2, as a
    fused environment over the reduced legs (k1, 1, 1 | k2, 1, 1)."""
    Nkb = env_matrix(N, dims1, dims2)
    E1, E2 = Q1.shape[0], Q2.shape[0]
    k1, k2 = Q1.shape[1], Q2.shape[1]
    N4 = Nkb.reshape(E1, E2, E1, E2)
    Nr = np.einsum("abcd,ak,bl,cm,dn->klmn", N4, Q1, Q2, Q1.conj(), Q2.conj())
    return np.transpose(Nr, (0, 2, 1, 3)).reshape(k1 * k1, 1, 1, k2 * k2, 1, 1)


def _as_site(r, s):
    """r[p, k, bond] as a four-slot tensor: the bond at slot s, the other
    slots (k, 1, 1) in slot order."""
    d, k, Db = r.shape
    return _insert(r.reshape(d, k, 1, 1, Db), s)


def _restore(t_like, Q, a, s):
    """t' = Q r' with the tensor laid out like t_like."""
    ra = _open(a, s)                                  # [p, k, bond]
    return _close(np.einsum("ek,pkb->peb", Q, ra), t_like, s)


def als_reduced(t1, t2, s1, s2, N, dims1, dims2, G, D, max_sweeps: int = 50, tol: float = 1e-13):
    """ALS on the reduced environment (the variant the thesis runs, Sec. 3.2):
    both site tensors split by reduce_site, ALS (same steps as als) on the
    reduced tensors r1, r2 with the projected environment, then t' = Q r'."""
    Q1, r1 = reduce_site(t1, s1)
    Q2, r2 = reduce_site(t2, s2)
    Nf = reduced_env(N, dims1, dims2, Q1, Q2)
    a, b, hist = als(_as_site(r1, s1), _as_site(r2, s2), s1, s2, Nf, [Q1.shape[1], 1, 1], [Q2.shape[1], 1, 1],
                     G, D, max_sweeps, tol)
    return _restore(t1, Q1, a, s1), _restore(t2, Q2, b, s2), hist


def bond_update(bbp: BlockBP, g1: int, k1: int, G, D: int, max_sweeps: int = 50, reduced: bool = False):
    """One ITE update of the bond leaving site g1 through slot k1, with the Edge
    TN of the converged messages of ``bbp``.  Returns (g2, new t_g1, new t_g2,
    Phi history); the tensors have the open legs of the lattice cut to 1."""
    coords, key1, key2 = bbp.bond_region(g1, k1)
    env = CoreEnv(bbp, coords, [key1, key2])
    N, labels, slots = env.edge(key1, key2)
    rs1, rs2 = env.sites[key1], env.sites[key2]
    joint = set(rs1.labels) & set(rs2.labels)
    s1 = rs1.labels.index(next(iter(joint)))
    s2 = rs2.labels.index(next(iter(joint)))
    t1, t2 = bbp.tc[rs1.gid], bbp.tc[rs2.gid]
    dims1 = [t1.shape[1 + s] for s in range(4) if s != s1]
    dims2 = [t2.shape[1 + s] for s in range(4) if s != s2]
    a, b, hist = (als_reduced if reduced else als)(t1, t2, s1, s2, N, dims1, dims2, G, D, max_sweeps)
    return rs2.gid, a, b, hist


def _put(t_full: np.ndarray, g: int, small: np.ndarray):
    """Write a tensor whose open legs are cut to 1 back into the full array."""
    t_full[g] = 0.0
    t_full[g][tuple(slice(0, n) for n in small.shape)] = small / np.abs(small).max()


def full_ite(geom, t: np.ndarray, chi: int, dts, edge_mats, h=None, bp_tol: float = 1e-10,
             bp_iter: int = 40, als_sweeps: int = 50, on_step=None, reduced: bool = False):
    """Alg. 2 (Full ITE using BlockBP) on a finite or periodic network: for
    every dt, every bond is updated with exp(-dt/2 h), forwards through the
    bond list and then backwards (second-order splitting); BlockBP runs to
    tol before every update, starting from the previous messages.  Returns
    the final tensors and the energy per site after each dt."""
    t = np.array(t, dtype=np.complex128)
    D = t.shape[2]
    h = heisenberg_h() if h is None else h
    bonds = list(geom.bonds())
    msgs = None
    energies = []

    def converged():
        nonlocal msgs
        bbp = BlockBP(geom, t, chi)
        bbp.init_messages(edge_mats)
        if msgs is not None:
            bbp.msgs = dict(msgs)
        bbp.run(bp_tol, bp_iter)
        msgs = dict(bbp.msgs)
        return bbp

    for dt in dts:
        G = gate(h, 0.5 * dt)
        for (g1, k1, _, _) in bonds + bonds[::-1]:
            bbp = converged()
            g2, a, b, _ = bond_update(bbp, g1, k1, G, D, als_sweeps, reduced)
            _put(t, g1, a)
            _put(t, g2, b)
        e = converged().energy_per_site()
        energies.append(e)
        if on_step is not None:
            on_step(dt, e)
    return t, energies


def full_ite_unit_cell(geom, t_cell: np.ndarray, chi: int, dts, edge_mats, h=None, bp_tol: float = 1e-10,
                       bp_iter: int = 40, als_sweeps: int = 50, on_step=None, reduced: bool = False):
    """Alg. 2 for a translation-invariant Kagome PEPS (Sec. 3.3): every site of
    type t (A, B, C) carries the unit cell's tensor t_cell[t]; each time step
    updates the six bonds of the unit cell (the up-triangle and the
    down-triangle through it, a mode of block 0, forwards then backwards,
    half steps), each on its bond inside the mode with the Edge TN of the
    converged messages, and writes the two new tensors into every site of
    their types.  Returns (t_cell, energy per site after each step)."""
    from .core import kagome_mode
    t_cell = np.array(t_cell, dtype=np.complex128)
    D = t_cell.shape[2]
    h = heisenberg_h() if h is None else h
    lat = geom.lattice
    b0 = geom.blocks[0]
    mode = next(m for (t, i, j) in b0.sites for v in range(3)
                for m in [kagome_mode(geom, 0, (i, j), v)] if m is not None)
    bonds = []
    for x in range(5):
        for k in range(4):
            t_, i, j = b0.sites[mode[x]]
            t2, i2, j2, _ = lat.neighbour(t_, i, j, k)
            if (t2, i2, j2) in [b0.sites[q] for q in mode[x + 1:]]:
                bonds.append((b0.gids[mode[x]], k))
    msgs = None
    energies = []

    def full():
        return np.array([t_cell[g % 3] for g in range(geom.n_sites)])

    def converged():
        nonlocal msgs
        bbp = BlockBP(geom, full(), chi)
        bbp.init_messages(edge_mats)
        if msgs is not None:
            bbp.msgs = dict(msgs)
        bbp.run(bp_tol, bp_iter)
        msgs = dict(bbp.msgs)
        return bbp

    for dt in dts:
        G = gate(h, 0.5 * dt)
        for (g1, k1) in bonds + bonds[::-1]:
            bbp = converged()
            g2, a, b, _ = bond_update(bbp, g1, k1, G, D, als_sweeps, reduced)
            for g, x in ((g1, a), (g2, b)):
                tmp = np.zeros((1,) + t_cell.shape[1:], dtype=np.complex128)
                _put(tmp, 0, x)
                t_cell[g % 3] = tmp[0]
        e = converged().energy_per_site()
        energies.append(e)
        if on_step is not None:
            on_step(dt, e)
    return t_cell, energies
