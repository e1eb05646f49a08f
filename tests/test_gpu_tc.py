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


def tc_gemm_tile(A, Bt, bf16, bn, group_m):
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
    P.bbp_k_tc_gemm_tile(bf16, Ad, ld, Bd, ld, C, N, M, N, K, 1.0, bn, group_m, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0, "pipeline wait timed out"
    return C.cpu().double()


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("M,N,K", [(300, 130, 1000), (1000, 600, 512), (2592, 520, 264), (17, 300, 40)])
def test_tc_gemm_tiles(M, N, K, bf16):
    """Every tile (bn 64 / 128 / 256, group_m 1 / 8 / 16) computes the same
    GEMM: each output element accumulates the same K steps in the same order
    whatever the tile, so the tiles agree to FP32 rounding (in practice
    bitwise), and each is within the operand-rounding bound of the FP64
    product."""
    g = torch.Generator().manual_seed(M + 3 * N + 7 * K)
    A = torch.randn(M, K, generator=g, dtype=torch.float64)
    Bt = torch.randn(N, K, generator=g, dtype=torch.float64)
    ref = A @ Bt.T
    scale = (A.abs() @ Bt.abs().T).max().item()
    u = 2.0 ** -8 if bf16 else 2.0 ** -11
    base = tc_gemm(A, Bt, bf16)
    same = 0
    for bn in (64, 128, 256):
        for gm in (1, 8, 16):
            C = tc_gemm_tile(A, Bt, bf16, bn, gm)
            assert (C - ref).abs().max().item() <= 2.5 * u * scale
            d = (C - base).abs().max().item()
            assert d <= 1e-6 * scale, f"bn={bn} group_m={gm}: {d:.3e}"
            same += int(d == 0.0)
    print(f"M={M} N={N} K={K} bf16={bf16}: {same} of 9 tiles bitwise equal to the default")


def test_autotune_record_run_load(tmp_path):
    """Recording the tensor-core shapes of a TF32 iteration, tuning them and
    reloading the cache: the table round-trips, the tuned iteration is
    recaptured (generation advances) and gives the same messages."""
    import synthetic as syn
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, 4, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(len(nb), 4, seed=7)

    def run(iters):
        ctx = P.bbp_create_peps(P.KAGOME, 6, 2, 1, 2, 4, t)
        P.bbp_partition_blocks(ctx, 2, 2)
        P.bbp_set_options(ctx, 32, P.TF32)
        P.bbp_init_messages(ctx, em)
        P.bbp_iterate(ctx, 0.0, iters)
        out = [np.concatenate([x.ravel() for x in P.bbp_get_message(ctx, b, f)]) for b in range(3) for f in range(4)]
        P.bbp_destroy(ctx)
        return out

    P.bbp_autotune_clear()
    P.bbp_autotune_record(True)
    before = run(3)
    P.bbp_autotune_record(False)
    _, pending, gen0 = P.bbp_autotune_info()
    assert pending >= 1, "no tensor-core GEMM was recorded"
    cache = str(tmp_path / "tiles.txt")
    tuned = P.bbp_autotune_run(cache)
    entries, pending2, gen1 = P.bbp_autotune_info()
    assert tuned == pending and entries == tuned and pending2 == 0 and gen1 > gen0
    lines = [ln for ln in open(cache) if ln.startswith("tc ")]
    assert len(lines) == entries
    P.bbp_autotune_clear()
    assert P.bbp_autotune_load(cache) == entries
    after = run(3)
    worst = max(float(np.abs(a - b).max()) for a, b in zip(before, after))
    print(f"autotune: {entries} shapes; largest message change after retuning {worst:.2e}")
    assert worst <= 1e-6
    P.bbp_autotune_clear()
