"""Kernel-level parity on the GPU: fusion (K1), truncated SVD (K3), QR.

Each CUDA kernel is called through the C ABI on device buffers and compared
element by element with the oracle (fusion) or with the mathematics the
kernel must reproduce (Eckart-Young truncation, QR factorisation).
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import tn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("D,n,perm,with_op", [
    (2, (2, 2, 2, 2), (0, 1, 2, 3), False),
    (3, (3, 1, 3, 3), (2, 0, 3, 1), False),
    (2, (1, 2, 2, 1), (3, 2, 1, 0), True),
    (4, (4, 4, 4, 4), (1, 3, 0, 2), True),
])
def test_fuse_matches_oracle(D, n, perm, with_op):
    d = 2
    t = syn.gaussian_peps(1, d, D, seed=3)[0]
    op = (np.random.default_rng(4).standard_normal((d, d)) + 1j * np.random.default_rng(5).standard_normal((d, d)))
    tt = dev(t)
    T = torch.zeros(int(np.prod([n[q] ** 2 for q in range(4)])), dtype=torch.complex128, device="cuda")
    P.bbp_k_fuse(tt, d, D, n, dev(op) if with_op else None, perm, T)
    got = host(T).reshape([n[p] ** 2 for p in perm])
    sl = (slice(None),) + tuple(slice(0, n[q]) for q in range(4))
    want = tn.fuse(t[sl], op if with_op else None).transpose(perm)
    assert np.abs(got - want).max() <= 1e-14 * max(1.0, np.abs(want).max())


def _gapped(m, n, seed, decay=0.7):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    s = decay ** np.arange(k) * (1.0 + 0.1 * rng.random(k))
    s = np.sort(s)[::-1]
    return (U * s) @ V.conj().T, s


@pytest.mark.parametrize("m,n,chi", [(12, 9, 4), (9, 12, 4), (16, 64, 8), (64, 16, 8), (200, 40, 32),
                                     (256, 256, 32), (512, 512, 32), (1024, 512, 32), (5, 5, 8)])
def test_svd_trunc_is_optimal_truncation(m, n, chi):
    Z, s = _gapped(m, n, seed=m * 7 + n)
    k = min(chi, m, n)
    Zd = dev(Z)
    U = torch.zeros(m * k, dtype=torch.complex128, device="cuda")
    R = torch.zeros(k * n, dtype=torch.complex128, device="cuda")
    work = torch.zeros(P.bbp_k_svd_work_bytes(m, n) // 16 + 16, dtype=torch.complex128, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.bbp_k_svd_trunc(Zd, m, n, chi, U, R, work, status)
    Uh, Rh = host(U).reshape(m, k), host(R).reshape(k, n)
    assert int(status.cpu()[0]) == 0
    # U is an isometry
    assert np.abs(Uh.conj().T @ Uh - np.eye(k)).max() < 1e-12
    # U Rem is the best rank-k approximation (Eckart-Young), unique for a gapped spectrum
    u, ss, vh = np.linalg.svd(Z, full_matrices=False)
    best = (u[:, :k] * ss[:k]) @ vh[:k]
    assert np.abs(Uh @ Rh - best).max() < 1e-12 * ss[0]
    assert np.allclose(np.linalg.norm(Rh, axis=1), ss[:k], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("m,n", [(10, 4), (4, 10), (7, 7), (512, 32), (1024, 32), (32, 512)])
def test_qr(m, n):
    rng = np.random.default_rng(m + 3 * n)
    A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    k = min(m, n)
    Ad = dev(A)
    Q = torch.zeros(m * k, dtype=torch.complex128, device="cuda")
    R = torch.zeros(k * n, dtype=torch.complex128, device="cuda")
    tau = torch.zeros(k + 1, dtype=torch.complex128, device="cuda")
    P.bbp_k_qr(Ad, m, n, Q, R, tau)
    Qh, Rh = host(Q).reshape(m, k), host(R).reshape(k, n)
    assert np.abs(Qh @ Rh - A).max() < 1e-12 * np.abs(A).max()
    assert np.abs(Qh.conj().T @ Qh - np.eye(k)).max() < 1e-13
    assert np.abs(np.tril(Rh, -1)).max() == 0.0
