"""Learning step (damping) and Hermitisation of BlockBP messages (test
infrastructure only).

Sec. "BlockBP Learning-step", Eq. of the learning step: the message that
replaces msg_old is msg_learned = alpha msg_new + (1 - alpha) msg_old,
alpha in [0, 1], summed as MPSs.  Sec. "Hermitize MPSs": a message is a
double-legged (ket, bra) MPS, i.e. an operator; its Hermitian part
B = (A + A^dagger) / 2 is formed by unfusing each leg into (ket, bra),
transposing to (bra, ket), conjugating, refusing and adding.

Readings (the thesis leaves these open):
* N: MPSs are added by the direct sum (bonds add, Sec. on MPS addition of
  the cited review) and the sum is compressed back to bond chi by a
  left-canonical QR sweep followed by a right-to-left truncated-SVD sweep
  that keeps min(chi, rows, cols) values at every cut; the result is then
  normalised as every message is (reading A).
* O: when both are used, the new message is Hermitised first and the
  learning step mixes the Hermitised message with the old one; the
  convergence distance is that of the message that replaces the old one.
"""
from __future__ import annotations

import numpy as np

from . import tn


def mps_add(A: list, B: list, a: complex = 1.0, b: complex = 1.0) -> list:
    """a A + b B as one MPS (direct sum of the bond spaces)."""
    k = len(A)
    if k != len(B):
        raise ValueError("MPS lengths differ")
    if k == 1:
        return [a * A[0] + b * B[0]]
    out = []
    for q in range(k):
        x, y = A[q], B[q]
        if q == 0:
            out.append(np.concatenate([a * x, b * y], axis=2))
        elif q == k - 1:
            out.append(np.concatenate([x, y], axis=0))
        else:
            lx, p, rx = x.shape
            ly, _, ry = y.shape
            t = np.zeros((lx + ly, p, rx + ry), dtype=np.complex128)
            t[:lx, :, :rx] = x
            t[lx:, :, rx:] = y
            out.append(t)
    return out


def mps_compress(A: list, chi: int, discarded: list | None = None) -> list:
    """Compress to bond chi (reading N): left-canonical QR sweep, then
    truncated SVDs from the right.  The singular values dropped at each cut
    are appended to `discarded` when given."""
    A = [np.array(a, dtype=np.complex128) for a in A]
    k = len(A)
    for q in range(k - 1):
        A[q], A[q + 1] = tn.qr_right(A[q], A[q + 1])
    for q in range(k - 1, 0, -1):
        l, p, r = A[q].shape
        U, s, Vh = np.linalg.svd(A[q].reshape(l, p * r), full_matrices=False)
        kk = min(chi, len(s))
        if discarded is not None:
            discarded.append(s[kk:])
        A[q] = Vh[:kk].reshape(kk, p, r)
        A[q - 1] = np.tensordot(A[q - 1], U[:, :kk] * s[:kk], axes=(2, 0))
    return A


def mps_dagger(A: list, dims: list) -> list:
    """The message read as an operator and Hermitian-conjugated: each fused
    leg ket * D + bra becomes bra * D + ket, and every entry is conjugated."""
    out = []
    for a, D in zip(A, dims):
        l, p, r = a.shape
        t = a.reshape(l, D, D, r).transpose(0, 2, 1, 3).reshape(l, p, r)
        out.append(np.conj(t))
    return out


def hermitise(A: list, dims: list, chi: int) -> list:
    """(A + A^dagger) / 2 compressed to bond chi (Sec. "Hermitize MPSs")."""
    return mps_compress(mps_add(A, mps_dagger(A, dims), 0.5, 0.5), chi)


def learned(new: list, old: list, alpha: float, chi: int) -> list:
    """alpha new + (1 - alpha) old compressed to bond chi (Eq. of the
    learning step, reading N)."""
    if alpha == 1.0:
        return [np.array(a) for a in new]
    return mps_compress(mps_add(new, old, alpha, 1.0 - alpha), chi)
