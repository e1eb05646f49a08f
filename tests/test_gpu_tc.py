"""K2 on the tensor cores: the tcgen05 GEMM and the split-precision complex
absorb, against plain PyTorch references of the same operation.

TF32 keeps 10 explicit mantissa bits (unit roundoff 2^-11), BF16 keeps 7
(2^-8); a K-term dot product of rounded operands then differs from the exact
one by at most about 2 u sum_k |a_k b_k| (FP32 accumulation adds K 2^-24).
The split absorb (hi*hi + hi*lo + lo*hi) leaves only the lo*lo term and the
rounding of lo, about 3 u^2 sum |a b| (~1e-6 for TF32), plus the FP32
accumulation of 6P terms (typically sqrt(6P) 2^-24 sum |a b|).
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


def tc_gemm(A, Bt, bf16):
    M, K = A.shape
    N = Bt.shape[0]
    step = 8 if bf16 else 4
    ld = (K + step - 1) // step * step
    dt = torch.bfloat16 if bf16 else torch.float32
    Ad = torch.zeros(M, ld, dtype=dt, device="cuda")
    Bd = torch.zeros(N, ld, dtype=dt, device="cuda")
    Ad[:, :K] = A.to("cuda", dt)
    Bd[:, :K] = Bt.to("cuda", dt)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.bbp_k_tc_gemm(bf16, Ad, ld, Bd, ld, C, N, M, N, K, 1.0, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0, "pipeline wait timed out"
    return C.cpu().double()


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 64, 64), (256, 256, 512), (200, 72, 100), (300, 130, 1000),
                                   (17, 5, 8)])
def test_tc_gemm(M, N, K, bf16):
    g = torch.Generator().manual_seed(M * 7919 + N * 31 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float64)
    Bt = torch.randn(N, K, generator=g, dtype=torch.float64)
    C = tc_gemm(A.float(), Bt.float(), bf16)
    # reference on the operands as the tensor core sees them
    if bf16:
        Ar, Br = A.to(torch.bfloat16).double(), Bt.to(torch.bfloat16).double()
        u = 2.0 ** -8
    else:
        Ar, Br = A.float().double(), Bt.float().double()
        u = 2.0 ** -11
    ref = Ar @ Br.T
    bound = (2 * u + K * 2.0 ** -24) * (Ar.abs() @ Br.abs().T)
    assert torch.isfinite(C).all()
    excess = ((C - ref).abs() - bound).max().item()
    print(f"M={M} N={N} K={K} bf16={bf16}: max |err| {(C - ref).abs().max().item():.3e}")
    assert excess <= 0.0
    if bf16:
        # bf16 operands: the exact product of the rounded operands, to FP32 accumulation
        acc = (C - ref).abs() <= K * 2.0 ** -20 * (Ar.abs() @ Br.abs().T) + 1e-30
        assert acc.all()


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("c64", [False, True])
@pytest.mark.parametrize("Pd,Q,l,r", [(256, 256, 32, 32), (16, 64, 8, 5), (36, 100, 3, 64)])
def test_tc_absorb(Pd, Q, l, r, bf16, c64):
    rng = np.random.default_rng(Pd + Q + l + r)
    X = rng.standard_normal((Pd, Q)) + 1j * rng.standard_normal((Pd, Q))
    S = (rng.standard_normal((l, Pd, r)) + 1j * rng.standard_normal((l, Pd, r))) * 1e-3
    ref = np.einsum("pq,apr->aqr", X, S)
    ct = torch.complex64 if c64 else torch.complex128
    Xd = torch.from_numpy(X).to("cuda", ct)
    Sd = torch.from_numpy(S).to("cuda", ct)
    Rd = torch.zeros(l, Q, r, dtype=ct, device="cuda")
    work = torch.zeros(P.bbp_k_tc_absorb_bytes(bf16, Pd, Q, l, r), dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.bbp_k_tc_absorb(bf16, c64, Xd, Pd, Q, Sd, l, r, Rd, work, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    R = Rd.cpu().numpy().astype(np.complex128)
    scale = np.einsum("pq,apr->aqr", np.abs(X), np.abs(S))
    rel = np.max(np.abs(R - ref) / scale)
    print(f"absorb P={Pd} Q={Q} l={l} r={r} bf16={bf16} c64={c64}: max err / sum|x s| = {rel:.2e}")
    # three-product split: ~3 u^2, plus FP32 accumulation over 6P terms
    assert rel < (3e-4 if bf16 else 2e-5)
