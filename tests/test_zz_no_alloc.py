"""The allocation-free SVD entry point (bbp_k_svd_trunc_noalloc).

It exists for callers that cannot allocate device memory when they need the
SVD (real-time loops that must not enter the allocator, hosts whose device
memory belongs to another runtime).  It must give the same
result as bbp_k_svd_trunc, which takes caller-allocated scratch, on two calls
in a row (the second one reusing the shared device array), and reject sizes
beyond its fixed scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def _matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    s = np.sort(0.8 ** np.arange(k) * (1 + 0.1 * rng.random(k)))[::-1]
    return (U * s) @ V.conj().T


def _run(fn, Z, m, n, chi, with_work):
    k = min(chi, m, n)
    U = torch.full((m * k,), complex(7, 7), dtype=torch.complex128, device="cuda")
    R = torch.full((k * n,), complex(7, 7), dtype=torch.complex128, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    if with_work:
        work = torch.zeros(P.bbp_k_svd_work_bytes(m, n) // 16 + 16, dtype=torch.complex128, device="cuda")
        fn(Z, m, n, chi, U, R, work, st)
    else:
        fn(Z, m, n, chi, U, R, st)
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == 0
    return U.cpu().numpy().reshape(m, k), R.cpu().numpy().reshape(k, n)


@pytest.mark.parametrize("m,n,chi", [(512, 512, 32), (40, 96, 8), (96, 40, 8)])
def test_noalloc_matches_allocating_entry_point(m, n, chi):
    for call, seed in enumerate((11, 12)):           # two calls in a row
        Z = torch.from_numpy(_matrix(m, n, seed + m)).cuda()
        U0, R0 = _run(P.bbp_k_svd_trunc, Z, m, n, chi, True)
        U1, R1 = _run(P.bbp_k_svd_trunc_noalloc, Z, m, n, chi, False)
        scale = np.abs(U0 @ R0).max()
        assert np.abs(U1 @ R1 - U0 @ R0).max() < 1e-12 * scale, f"call {call}"
        assert np.allclose(np.linalg.norm(R1, axis=1), np.linalg.norm(R0, axis=1), rtol=1e-12, atol=1e-14)
        k = U1.shape[1]
        assert np.abs(U1.conj().T @ U1 - np.eye(k)).max() < 1e-12


def test_noalloc_rejects_oversized():
    m = n = 1024
    Z = torch.zeros(m * n, dtype=torch.complex128, device="cuda")
    U = torch.zeros(m * 8, dtype=torch.complex128, device="cuda")
    R = torch.zeros(8 * n, dtype=torch.complex128, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(P.BBPError) as ei:
        P.bbp_k_svd_trunc_noalloc(Z, m, n, 8, U, R, st)
    assert ei.value.status == 1
    assert "scratch" in str(ei.value)
