// Host-side launchers of the BlockBP CUDA kernels (sm_103a).
// Complex numbers are interleaved (re, im): double2 (complex128, the FP64
// path) or float2 (complex64, the mixed path).  Launchers are overloaded on
// the element type; norms, log-scales and message distances are double.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace bbp {

// K1: double-layer fusion (Sec. 1.2 / Sec. 2.1), optionally with a d x d
// operator O inserted: T = sum_{s,s'} O[s,s'] t[s', ket] conj(t[s, bra]),
// evaluated in complex128 and stored in the output type.
// t: [d][Dfull]^4 site tensor; n[k] in {1, Dfull} is the used extent of leg k
// (1 on an open boundary, index 0); out axis q is source leg perm[q]; fused
// index ket * n + bra.  op may be null (identity).
cudaError_t launch_fuse(const double2* t, int d, int Dfull, const int n[4], const double2* op, const int perm[4],
                        double2* T, cudaStream_t s);
cudaError_t launch_fuse(const double2* t, int d, int Dfull, const int n[4], const double2* op, const int perm[4],
                        float2* T, cudaStream_t s);

// Complex GEMM, row-major: C[b] = alpha * opA(A[b]) * opB(B[b]) + beta * C[b].
// op: 'N' as stored, 'T' transposed, 'C' conjugate-transposed.
cudaError_t launch_zgemm(char opA, char opB, int M, int N, int K, double2 alpha, const double2* A, int lda,
                         long long strideA, const double2* B, int ldb, long long strideB, double2 beta,
                         double2* C, int ldc, long long strideC, int batch, cudaStream_t s);
cudaError_t launch_zgemm(char opA, char opB, int M, int N, int K, float2 alpha, const float2* A, int lda,
                         long long strideA, const float2* B, int ldb, long long strideB, float2 beta, float2* C,
                         int ldc, long long strideC, int batch, cudaStream_t s);

// Opt-in of large dynamic shared memory for every staged kernel on the
// current device; call once before any stream capture.
cudaError_t init_kernel_attributes();
cudaError_t init_tc_attributes();

// Householder QR of A (m x n, row-major, overwritten): Q (m x k), R (k x n),
// k = min(m, n).  tau: k complex scratch.  One CTA per matrix.
cudaError_t launch_qr(double2* A, int m, int n, double2* Q, double2* R, double2* tau, cudaStream_t s);
cudaError_t launch_qr(float2* A, int m, int n, float2* Q, float2* R, float2* tau, cudaStream_t s);

// R factor only of A (m x n, row-major, not modified): k x n, k = min(m, n),
// upper triangular with a real diagonal.  Tall inputs are split into row
// blocks whose R's are stacked and factorised again; s0, s1: scratch of
// m * n elements each.  Panels too wide for that (n x n beyond shared memory,
// or row blocks shorter than 2n) are factorised by one CTA over a copy in s0.
cudaError_t launch_qr_r(const double2* A, int m, int n, double2* R, double2* s0, double2* s1, cudaStream_t s);
cudaError_t launch_qr_r(const float2* A, int m, int n, float2* R, float2* s0, float2* s1, cudaStream_t s);

// Truncated SVD Z (m x n) = U S V^H keeping k = min(chi, m, n) triplets with
// the largest singular values: writes U (m x k) and Rem = S V^H (k x n).
// complex128: exact one-sided (row) Jacobi.  complex64: Jacobi when
// min(m, n) <= rand_block(m, n, chi), else a randomised subspace iteration
// with `power_iters` power steps reduces Z to rand_block rows first.
// *status is set to 1 if a sweep limit was reached (never cleared).
size_t svd_work_bytes(int m, int n);
// complex64: with tensor_cores the range-finder products of the randomised
// path run on tcgen05 (split TF32) and the scratch includes their packed
// operands.
size_t svd_work_bytes_c64(int m, int n, int chi, bool tensor_cores = false);
// Scratch bound for every complex64 split with min(m, n) <= max_min and max(m, n) <= max_max.
size_t svd_work_bound_c64(int max_min, int max_max, int chi, bool tensor_cores = false);
int rand_block(int m, int n, int chi);
cudaError_t launch_svd_trunc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work,
                             int* status, cudaStream_t s);
cudaError_t launch_svd_trunc(const float2* Z, int m, int n, int chi, float2* U, float2* Rem, void* work, int* status,
                             cudaStream_t s, int power_iters, bool tensor_cores = false, int* tc_err = nullptr);
// complex128 randomised truncation (the engine's FP64 path): b = 2 chi
// directions, power_iters power steps (six by default), the b x b factor by
// complex128 Jacobi; small matrices (min(m, n) <= max(4 chi, 64)) take the
// exact Jacobi.
int rand_block64(int m, int n, int chi);
size_t svd_work_bytes_rand64(int m, int n, int chi);
size_t svd_work_bound_rand64(int max_min, int max_max, int chi);
cudaError_t launch_svd_trunc_rand64(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work,
                                    int* status, cudaStream_t s, int power_iters);
// Sweeps and rotations of the last complex128 launch_svd_trunc that used `work` (synchronises s).
cudaError_t svd_stats(const void* work, int m, int n, int* sweeps, long long* rotations, cudaStream_t s);

// Frobenius norm of a tensor: A /= ||A||, *logscale += log ||A|| (0 norm: logscale = -inf).
cudaError_t launch_normalise(double2* A, long long n, double* logscale, cudaStream_t s);
cudaError_t launch_normalise(float2* A, long long n, double* logscale, cudaStream_t s);

// Out-of-place copy with the (l, p, r) -> (r, p, l) transpose, or a plain copy.
cudaError_t launch_copy_tensor(const double2* src, double2* dst, int l, int p, int r, bool transpose, cudaStream_t s);
cudaError_t launch_copy_tensor(const float2* src, float2* dst, int l, int p, int r, bool transpose, cudaStream_t s);

cudaError_t launch_fill(double2* A, long long n, double re, double im, cudaStream_t s);
cudaError_t launch_fill(float2* A, long long n, double re, double im, cudaStream_t s);

// dst (cols x rows) = conj(src (rows x cols))^T
cudaError_t launch_conj_transpose(const double2* src, int rows, int cols, double2* dst, cudaStream_t s);
cudaError_t launch_conj_transpose(const float2* src, int rows, int cols, float2* dst, cudaStream_t s);
// dst = src (d0, d1, d2) with axes permuted: dst axis q is src axis perm[q]
cudaError_t launch_permute3(const double2* src, int d0, int d1, int d2, const int perm[3], double2* dst, cudaStream_t s);
cudaError_t launch_permute3(const float2* src, int d0, int d1, int d2, const int perm[3], float2* dst, cudaStream_t s);

// ITE helpers (k_ite.cu, complex128).  A strided view: over the row-major
// index space dims[0..rank), dst[sum c_q dstr[q]] = src[sum c_q sstr[q]]
// (permutations, gathers and scatters of small tensors).
constexpr int kStridedMaxRank = 12;
struct StridedView {
  int rank = 0;
  long long total = 0;
  long long dims[kStridedMaxRank], sstr[kStridedMaxRank], dstr[kStridedMaxRank];
};
cudaError_t launch_strided_copy(const double2* src, double2* dst, const StridedView& v, cudaStream_t s);
// W (n x ncols) rows scaled by 1 / |Rem row|^2, zero below (rcond sigma_max)^2:
// with M = U Rem the truncated SVD of a square M, Rem^H (this applied to
// U^H c) is the least-squares solution of M x = c.
cudaError_t launch_pinv_rows(double2* W, const double2* Rem, int n, int ncols, double rcond, cudaStream_t s);
// *out = Re sum T[e] conj(X[e])
cudaError_t launch_quad_form(const double2* T, const double2* X, long long n, double* out, cudaStream_t s);
// A /= max |A|
cudaError_t launch_scale_absmax(double2* A, long long n, cudaStream_t s);
// y += a x
cudaError_t launch_axpy(const double2* x, double2* y, long long n, double2 a, cudaStream_t s);

// An MPS passed to a kernel by value (no device-side tables, no copies).
constexpr int kMaxChain = 64;
struct ChainDesc {
  void* T[kMaxChain];
  int l[kMaxChain], p[kMaxChain], r[kMaxChain];
  int D[kMaxChain];   // bond dimension of each fused leg (leg index ket * D + bra)
  int k;
};

// K4, reading A: unit norm and <I|M> real positive, the chain products
// accumulated in complex128.  work: complex128 scratch of
// 2 * 64 * 64 + 64^3 + 256 entries.  One CTA.
cudaError_t launch_msg_normalise(const ChainDesc& m, bool c64, double2* work, cudaStream_t s);

// Convergence word of an iteration: out[0] = largest of dist[0..nu), the
// int after it = flags (1 non-finite, 2 sweep limit, 4 tensor-core timeout,
// 8 converged: largest <= *tol and no other flag); status: 2 ints per update.
cudaError_t launch_iter_reduce(const double* dist, const int* status, int nu, const double* tol, double* out,
                               cudaStream_t s);

// Direct-sum tensor of (new, -old) at chain position pos, in the input type.
cudaError_t launch_direct_sum(const double2* a, int la, int ra, const double2* b, int lb, int rb, int p, int pos,
                              int k, double2* out, cudaStream_t s);
cudaError_t launch_direct_sum(const float2* a, int la, int ra, const float2* b, int lb, int rb, int p, int pos, int k,
                              float2* out, cudaStream_t s);

// a x + b y (MPS addition by the direct sum, coefficients on the first
// tensor) at chain position pos of k; output (L, p, R) with L = lx (pos 0 or
// k == 1) else lx + ly, R = rx (pos k - 1 or k == 1) else rx + ry.
cudaError_t launch_mps_sum(const double2* x, int lx, int rx, const double2* y, int ly, int ry, int p, int pos, int k,
                           double2 a, double2 b, double2* out, cudaStream_t s);
cudaError_t launch_mps_sum(const float2* x, int lx, int rx, const float2* y, int ly, int ry, int p, int pos, int k,
                           double2 a, double2 b, float2* out, cudaStream_t s);
// Hermitian conjugate of a message tensor (l, D*D, r) as an operator.
cudaError_t launch_mps_dagger(const double2* src, int l, int D, int r, double2* dst, cudaStream_t s);
cudaError_t launch_mps_dagger(const float2* src, int l, int D, int r, float2* dst, cudaStream_t s);

// *dist = ||R||_F accumulated in double.
cudaError_t launch_frob(const double2* R, long long n, double* dist, cudaStream_t s);
cudaError_t launch_frob(const float2* R, long long n, double* dist, cudaStream_t s);

// Plain contraction of two MPS (no conjugation), accumulated in complex128.
cudaError_t launch_mps_dot(const ChainDesc& a, const ChainDesc& b, bool c64, double2* work, double2* out,
                           cudaStream_t s);

// K2 on tcgen05 (k_tc.cu): real GEMM C = alpha * A * Bt^T, A (M x K) and Bt
// (N x K) row-major in TF32 (fp32 storage) or BF16, C fp32; *err = 1 when a
// pipeline wait timed out.  The complex absorb R[a] = X^T S[a] runs as one
// split-precision real GEMM (hi*hi + hi*lo + lo*hi).
// algo_flops: the work the kernel timer credits to the launch (default the
// real GEMM's 2 M N K; the split-precision complex products pass their
// complex flops, 8 per complex multiply-add).
cudaError_t launch_tc_gemm(bool bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C,
                           long long ldc, int M, int N, int K, float alpha, int* err, cudaStream_t s,
                           double algo_flops = 0.0);
// The same GEMM with an explicit tile: bn in {64, 128, 256}, group_m >= 1.
cudaError_t launch_tc_gemm_tile(bool bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C,
                                long long ldc, int M, int N, int K, float alpha, int* err, cudaStream_t s, int bn,
                                int group_m, double algo_flops = 0.0);
// Tile autotuner of launch_tc_gemm (k_tc.cu): record collects the shapes of
// later launches that have no table entry; tc_autotune times the candidate
// tiles of each collected shape (synchronously, on its own stream, outside
// any capture) and writes the table to cache_path when it is not null;
// tc_autotune_load reads a table (returns the entries read, -1 when the file
// cannot be opened).  The generation counts table changes (captured graphs
// that launched with an older table are re-captured).
void tc_autotune_record(bool on);
cudaError_t tc_autotune(const char* cache_path, int* tuned);
int tc_autotune_load(const char* cache_path);
void tc_autotune_info(int* entries, int* pending);
void tc_autotune_clear();
unsigned long long tc_tune_generation();
size_t tc_absorb_bytes(bool bf16, int P, int Q, int l, int r);
cudaError_t launch_tc_absorb(bool bf16, const double2* X, int P, int Q, const double2* S, int l, int r, double2* R,
                             void* work, int* err, cudaStream_t s);
cudaError_t launch_tc_absorb(bool bf16, const float2* X, int P, int Q, const float2* S, int l, int r, float2* R,
                             void* work, int* err, cudaStream_t s);

// General complex64 GEMM on tcgen05 (k_tc.cu): C (M x N, row stride ldc
// complex) = op(A) (M x K) op(B) (K x N), as one split-precision real GEMM
// (hi*hi + hi*lo + lo*hi, FP32 accumulation) that writes C's interleaved
// (re, im) entries directly.  The operands are packed first into scratch of
// tc_zpack_bytes(bf16, M, K) (A) and tc_zpack_bytes(bf16, 2N, K) (B); op is
// 'N', 'T' or 'C' (A: M x K as stored, or stored K x M; B: K x N as stored, or
// stored N x K).  A packed operand may be reused by several products.
size_t tc_zpack_bytes(bool bf16, int rows, int K);
cudaError_t tc_zpack_a(bool bf16, char opA, int M, int K, const float2* A, long long lda, void* out, cudaStream_t s);
cudaError_t tc_zpack_b(bool bf16, char opB, int K, int N, const float2* B, long long ldb, void* out, cudaStream_t s);
cudaError_t tc_zgemm_packed(bool bf16, int M, int N, int K, const void* Ap, const void* Bp, float2* C, long long ldc,
                            int* err, cudaStream_t s);

// ALU peak microbenchmark (k_peak.cu): blocks x 256 threads, iters rounds of
// 8 independent FMA chains each; fma_peak_flops gives the flops launched.
double fma_peak_flops(bool fp64, int blocks, int iters);
cudaError_t launch_fma_peak(bool fp64, int blocks, int iters, void* out, cudaStream_t s);

// Live timing of one kernel class (ktimer.cpp): every launch of the selected
// class is bracketed by CUDA events on its stream; totals of launches,
// milliseconds and algorithmic flops accumulate until read.
enum KernelClass { KC_NONE = 0, KC_JACOBI = 1, KC_ORTH = 2, KC_QR = 3, KC_TC = 4, KC_ABSORB = 5, KC_GEMM = 6 };
void ktimer_select(int cls);
int ktimer_class();
double* ktimer_device_flops(int cls);        // device accumulator for kernels that count their own flops
void ktimer_set_tag(long long tag);          // tag of pairs recorded by this thread (-1: eager)
void ktimer_drop_tag(long long tag);
void ktimer_collect(long long tag);          // after a synchronise: add the pairs of `tag`
void ktimer_read(long long* n, double* ms, double* flops);
struct KTimerScope {
  KTimerScope(int cls, cudaStream_t s, double flops);
  ~KTimerScope();
  KTimerScope(const KTimerScope&) = delete;
  KTimerScope& operator=(const KTimerScope&) = delete;

 private:
  cudaStream_t s_ = nullptr;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool external_ = false;
};
// Complex Householder QR with the explicit Q, 8 real flops per complex
// multiply-add: 2 x 8 (2 a k^2 - 2 k^3 / 3), a = max(m, n), k = min(m, n).
inline double qr_flops(int m, int n) {
  const double a = m > n ? m : n, k = m < n ? m : n;
  return 16.0 * (2.0 * a * k * k - 2.0 * k * k * k / 3.0);
}

// Householder QR of tall panels on a cluster of up to kPanelMaxCluster CTAs
// (k_panel.cu): A (m x n, m >= n, row-major, not modified) = Q (m x n) R
// (n x n, upper triangular, real diagonal); Q or R may be null.  Q may alias
// A.  batch panels at a stride of `stride` elements (R at n * n).
// panel_cluster: the fewest CTAs whose shared memory holds an m x n panel of
// elem-byte entries (with the reflector scalars Q needs when want_q; 0 when
// even 16 do not); panel_cluster_auto: the cluster size of an automatic
// launch.  cluster = 0 picks it; a given size must be at least
// panel_cluster(m, n, elem) and at most kPanelMaxCluster.
constexpr int kPanelMaxCluster = 16;
int panel_cluster(int m, int n, size_t elem, bool want_q = true);
int panel_cluster_auto(int m, int n, size_t elem, bool want_q = true);
cudaError_t init_panel_attributes();
cudaError_t launch_panel_qr(const float2* A, int m, int n, float2* Q, float2* R, int batch, long long stride,
                            cudaStream_t s, int cluster = 0);
cudaError_t launch_panel_qr(const double2* A, int m, int n, double2* Q, double2* R, int batch, long long stride,
                            cudaStream_t s, int cluster = 0);
// Panels taller than one cluster holds (panel_cluster = 0): two-level TSQR
// over row chunks that each fit one cluster; Q is required, R may be null.
// panel_chunk_scratch_bytes: the device scratch it needs (0 when the panel
// fits one cluster or cannot be chunked).
size_t panel_chunk_scratch_bytes(int m, int n, size_t elem);
cudaError_t launch_panel_qr_chunked(const float2* A, int m, int n, float2* Q, float2* R, void* scratch,
                                    cudaStream_t s);
cudaError_t launch_panel_qr_chunked(const double2* A, int m, int n, double2* Q, double2* R, void* scratch,
                                    cudaStream_t s);

// Allocation-free truncated SVD (k_noalloc.cu): scratch in a fixed device
// array of noalloc_scratch_bytes(); *too_large is set when svd_work_bytes(m, n)
// exceeds it (nothing is launched then).
size_t noalloc_scratch_bytes();
cudaError_t launch_svd_trunc_noalloc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, int* status,
                                     cudaStream_t s, bool* too_large);

}  // namespace bbp
