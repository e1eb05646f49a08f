// Host-side launchers of the BlockBP CUDA kernels (sm_103a).
// Complex numbers are interleaved (re, im) doubles (double2) unless noted.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace bbp {

// K1: double-layer fusion (Sec. 1.2 / Sec. 2.1), optionally with a d x d
// operator O inserted: T = sum_{s,s'} O[s,s'] t[s', ket] conj(t[s, bra]).
// t: [d][Dfull]^4 site tensor; n[k] in {1, Dfull} is the used extent of leg k
// (1 on an open boundary, index 0); out axis q is source leg perm[q]; fused
// index ket * n + bra.  op may be null (identity).
cudaError_t launch_fuse(const double2* t, int d, int Dfull, const int n[4], const double2* op,
                        const int perm[4], double2* T, cudaStream_t s);

// Complex FP64 GEMM, row-major: C[b] = alpha * opA(A[b]) * opB(B[b]) + beta * C[b].
// op: 'N' as stored, 'T' transposed, 'C' conjugate-transposed.
cudaError_t launch_zgemm(char opA, char opB, int M, int N, int K, double2 alpha, const double2* A, int lda,
                         long long strideA, const double2* B, int ldb, long long strideB, double2 beta,
                         double2* C, int ldc, long long strideC, int batch, cudaStream_t s);

// Householder QR of A (m x n, row-major, overwritten): Q (m x k), R (k x n),
// k = min(m, n).  tau: k complex scratch.  One CTA per matrix.
cudaError_t launch_qr(double2* A, int m, int n, double2* Q, double2* R, double2* tau, cudaStream_t s);

// Truncated SVD by one-sided (row) Jacobi: Z (m x n) = U S V^H, keep
// k = min(chi, m, n) triplets with the largest singular values.
// Writes U (m x k) and Rem = S V^H (k x n).  Z is read only.
// work must hold svd_work_bytes(m, n); *status is set to 1 if the sweep limit
// was reached (left untouched otherwise, so callers clear it once).
size_t svd_work_bytes(int m, int n);
cudaError_t launch_svd_trunc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work,
                             int* status, cudaStream_t s);
// Sweeps and rotations of the last launch_svd_trunc that used `work` (synchronises s).
cudaError_t svd_stats(const void* work, int m, int n, int* sweeps, long long* rotations, cudaStream_t s);

// Frobenius norm of a tensor: A /= ||A||, *logscale += log ||A|| (0 norm: logscale = -inf).
cudaError_t launch_normalise(double2* A, long long n, double* logscale, cudaStream_t s);

// Out-of-place copy with the (l, p, r) -> (r, p, l) transpose, or a plain copy.
cudaError_t launch_copy_tensor(const double2* src, double2* dst, int l, int p, int r, bool transpose, cudaStream_t s);

// Fill with ones / zero.
cudaError_t launch_fill(double2* A, long long n, double re, double im, cudaStream_t s);

// Message finalisation (K4, reading A): unit norm and <I|M> real positive.
// tensors: k device pointers with shapes (l, p, r) on device; D: bond dimension
// of each fused leg (leg index ket * D + bra).  One CTA.
cudaError_t launch_msg_normalise(double2* const* tensors, const int* shapes, int k, const int* Dleg,
                                 double* work, cudaStream_t s);

// Build the direct-sum tensor of (new, -old) for the message distance sweep.
cudaError_t launch_direct_sum(const double2* a, int la, int ra, const double2* b, int lb, int rb, int p,
                              int pos, int k, double2* out, cudaStream_t s);

// out = ||R||_F of an (m x n) matrix into *dist.
cudaError_t launch_frob(const double2* R, long long n, double* dist, cudaStream_t s);

// Plain contraction of two MPS (no conjugation): value = sum prod A_q B_q.
// Writes the complex value to *out.  work: 2 * maxl * maxl complex.  One CTA.
cudaError_t launch_mps_dot(double2* const* A, double2* const* B, const int* shA, const int* shB, int k,
                           double2* work, double2* out, cudaStream_t s);

}  // namespace bbp

namespace bbp {
// dst (cols x rows) = conj(src (rows x cols))^T
cudaError_t launch_conj_transpose(const double2* src, int rows, int cols, double2* dst, cudaStream_t s);
// dst = src (d0, d1, d2) with axes permuted: dst axis q is src axis perm[q]
cudaError_t launch_permute3(const double2* src, int d0, int d1, int d2, const int perm[3], double2* dst, cudaStream_t s);
}  // namespace bbp

namespace bbp {
// Allocation-free truncated SVD (k_noalloc.cu): scratch in a fixed device
// array of noalloc_scratch_bytes(); *too_large is set when svd_work_bytes(m, n)
// exceeds it (nothing is launched then).
size_t noalloc_scratch_bytes();
cudaError_t launch_svd_trunc_noalloc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, int* status,
                                     cudaStream_t s, bool* too_large);
}  // namespace bbp
