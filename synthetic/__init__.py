"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers and lays them out in the documented input
formats; it holds none of the BlockBP arithmetic (no fusion, contraction,
truncation or message update).  Both implementations receive the same arrays.

Input formats (the same ones the C ABI documents in include/bbp.h):

* PEPS tensors: complex128 array ``[n_sites][d][D][D][D][D]``; the four
  virtual legs follow the per-lattice slot order below.
* Initial edge matrices: complex128 array ``[n_sites][4][D][D]``; entry
  ``[s][k]`` is the D x D positive semi-definite matrix that the initial
  (bond-1) incoming message places on leg slot ``k`` of site ``s``.  Only the
  slots that cross a block face are read.

Site numbering and leg slots
----------------------------
Square lattice ``Lx x Ly`` (open or periodic): site ``r*Lx + c`` for row ``r``
(0 = top) and column ``c`` (0 = left); slots ``(up, right, down, left)``.

Kagome lattice ``Lx x Ly`` unit cells with lattice vectors a1 (along x) and
a2 (60 degrees up): unit cell ``u = j*Lx + i`` holds sites ``3u+0 = A``,
``3u+1 = B = A + a1/2`` and ``3u+2 = C = A + a2/2``.  Slots:

* A(i,j): B(i,j), C(i,j), B(i-1,j), C(i,j-1)
* B(i,j): A(i,j), C(i,j), A(i+1,j), C(i+1,j-1)
* C(i,j): A(i,j), B(i,j), A(i,j+1), B(i-1,j+1)

(indices taken modulo the super-cell, which is always periodic).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "square_neighbours",
    "kagome_neighbours",
    "gaussian_peps",
    "normalise_sigma_max",
    "random_dimer_covering",
    "dimer_singlet_peps",
    "initial_edge_matrices",
    "pauli",
]


def square_neighbours(Lx: int, Ly: int, periodic: bool):
    """Neighbour table ``nb[s][k] = (s2, k2)`` or ``None`` on an open boundary."""
    nb = []
    for r in range(Ly):
        for c in range(Lx):
            row = []
            for (dr, dc, back) in ((-1, 0, 2), (0, 1, 3), (1, 0, 0), (0, -1, 1)):
                r2, c2 = r + dr, c + dc
                if periodic:
                    r2 %= Ly
                    c2 %= Lx
                if 0 <= r2 < Ly and 0 <= c2 < Lx:
                    row.append((r2 * Lx + c2, back))
                else:
                    row.append(None)
            nb.append(row)
    return nb


# (site type, slot) -> (neighbour type, di, dj, neighbour slot)
_KAGOME_SLOTS = {
    (0, 0): (1, 0, 0, 0), (0, 1): (2, 0, 0, 0), (0, 2): (1, -1, 0, 2), (0, 3): (2, 0, -1, 2),
    (1, 0): (0, 0, 0, 0), (1, 1): (2, 0, 0, 1), (1, 2): (0, 1, 0, 2), (1, 3): (2, 1, -1, 3),
    (2, 0): (0, 0, 0, 1), (2, 1): (1, 0, 0, 1), (2, 2): (0, 0, 1, 3), (2, 3): (1, -1, 1, 3),
}


def kagome_neighbours(Lx: int, Ly: int):
    """Neighbour table of the periodic Kagome super-cell of ``Lx x Ly`` unit cells."""
    nb = []
    for j in range(Ly):
        for i in range(Lx):
            for t in range(3):
                row = []
                for k in range(4):
                    t2, di, dj, k2 = _KAGOME_SLOTS[(t, k)]
                    i2, j2 = (i + di) % Lx, (j + dj) % Ly
                    row.append((3 * (j2 * Lx + i2) + t2, k2))
                nb.append(row)
    return nb


def _cgauss(rng: np.random.Generator, shape) -> np.ndarray:
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def normalise_sigma_max(t: np.ndarray) -> np.ndarray:
    """Divide each site tensor by its largest singular value as a d x D^4 matrix."""
    out = np.empty_like(t)
    for s in range(t.shape[0]):
        m = t[s].reshape(t.shape[1], -1)
        out[s] = t[s] / np.linalg.norm(m, 2)
    return out


def gaussian_peps(n_sites: int, d: int, D: int, seed: int, normalise: bool = True) -> np.ndarray:
    """I.i.d. complex Gaussian site tensors ``[n][d][D]^4`` (N(0,1) + i N(0,1))."""
    rng = np.random.default_rng(seed)
    t = _cgauss(rng, (n_sites, d, D, D, D, D))
    return normalise_sigma_max(t) if normalise else t


def random_dimer_covering(nb, seed: int):
    """Seeded random perfect matching of the lattice graph given by ``nb``.

    Returns a list ``partner[s] = (s2, k, k2)``: site s pairs with s2 through
    its slot k (slot k2 of s2).  Depth-first search with a seeded edge order.
    """
    n = len(nb)
    rng = np.random.default_rng(seed)
    order = [list(rng.permutation(4)) for _ in range(n)]
    partner = [None] * n

    def first_free():
        for s in range(n):
            if partner[s] is None:
                return s
        return -1

    def solve() -> bool:
        s = first_free()
        if s < 0:
            return True
        for k in order[s]:
            e = nb[s][k]
            if e is None:
                continue
            s2, k2 = e
            if s2 == s or partner[s2] is not None:
                continue
            partner[s] = (s2, k, k2)
            partner[s2] = (s, k2, k)
            if solve():
                return True
            partner[s] = None
            partner[s2] = None
        return False

    if not solve():
        raise ValueError("lattice has no perfect dimer covering")
    return partner


def dimer_singlet_peps(nb, d: int, D: int, seed: int, noise: float, noise_seed: int) -> np.ndarray:
    """Product of singlets on a random dimer covering, embedded in bond dimension D.

    For a dimer (s, s2) through slots (k, k2): t_s[p, leg k = a] = delta(p, a)
    and t_s2[p, leg k2 = a] = eps(a, p) / sqrt(2) with eps(0,1) = 1,
    eps(1,0) = -1, every other leg at index 0.  Contracting the shared leg
    gives the singlet (|01> - |10>)/sqrt(2).  Then ``noise`` times a complex
    Gaussian is added to every entry.
    """
    if d != 2 or D < 2:
        raise ValueError("singlet embedding needs d = 2 and D >= 2")
    n = len(nb)
    partner = random_dimer_covering(nb, seed)
    t = np.zeros((n, d, D, D, D, D), dtype=np.complex128)
    for s in range(n):
        s2, k, _ = partner[s]
        first = s < s2
        for p in range(2):
            for a in range(2):
                if first:
                    val = 1.0 if a == p else 0.0
                else:
                    val = (1.0 if (a, p) == (0, 1) else -1.0 if (a, p) == (1, 0) else 0.0) / np.sqrt(2.0)
                if val == 0.0:
                    continue
                idx = [0, 0, 0, 0]
                idx[k] = a
                t[(s, p) + tuple(idx)] = val
    if noise > 0.0:
        rng = np.random.default_rng(noise_seed)
        t = t + noise * _cgauss(rng, t.shape)
    return t


def initial_edge_matrices(n_sites: int, D: int, seed: int, eps: float = 0.1) -> np.ndarray:
    """Per-leg initial message matrices: identity plus a seeded PSD perturbation.

    ``m = I + eps * G G^dagger / ||G G^dagger||_F`` with G complex Gaussian.
    """
    rng = np.random.default_rng(seed)
    g = _cgauss(rng, (n_sites, 4, D, D))
    gg = g @ np.conj(np.swapaxes(g, -1, -2))
    nrm = np.linalg.norm(gg, axis=(-2, -1), keepdims=True)
    return np.eye(D)[None, None] + eps * gg / nrm


def pauli():
    """Pauli matrices (x, y, z) as complex128 2 x 2 arrays."""
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return sx, sy, sz
