// Complex kernels of the BlockBP message update (sm_103a), templated on the
// element type: complex128 (double2, the FP64 parity path) and complex64
// (float2, the mixed path).  Norms, log-scales and message distances
// accumulate in double in both.
//
//  K1 fuse           double-layer (ket-bra) tensor, Sec. 1.2 / Sec. 2.1
//  gemm              complex GEMM used for merges, contractions and gauge moves
//  qr                Householder QR (canonical-form moves, Sec. 2.3.3)
//  K3 svd_trunc      truncated SVD (Sec. 1.1.1, 1.1.3): one-sided (row) Jacobi;
//                    in complex64, large matrices are first reduced by a
//                    randomised subspace iteration and Jacobi runs on the
//                    small projected matrix
//  K4 msg_*          message normalisation, phase and distance
//
// Large Jacobi problems run on a thread-block cluster (one matrix per
// cluster, cluster barriers between rounds); every loop is bounded.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <atomic>
#include <cmath>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace bbp {

namespace {

template <typename C> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <typename C>
__host__ __device__ __forceinline__ C cx(double x, double y) {
  C r;
  r.x = (typename RealOf<C>::T)x;
  r.y = (typename RealOf<C>::T)y;
  return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {   // conj(a) * b
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) {
  a.x = a.x * (typename RealOf<C>::T)s;
  a.y = a.y * (typename RealOf<C>::T)s;
  return a;
}
template <typename C> __device__ __forceinline__ typename RealOf<C>::T cabs2(C a) { return a.x * a.x + a.y * a.y; }
template <typename C> __device__ __forceinline__ double cabs2d(C a) { return (double)a.x * a.x + (double)a.y * a.y; }
__device__ __forceinline__ double2 c128(double2 a) { return a; }
__device__ __forceinline__ double2 c128(float2 a) { return make_double2(a.x, a.y); }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double; result broadcast to all threads.
__device__ double block_sum(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (lane < nw) ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

// ------------------------------------------------------------------ K1 fuse
// One output entry per thread, consecutive threads writing consecutive
// entries.  The sum over the physical index runs in complex128 for a
// complex128 output and in complex64 for a complex64 output (two products
// per term: the rounding of the stored entry dominates either way); the
// operator, when present, is applied in complex128.  Index arithmetic in 32
// bits (D <= 8: at most 2^24 entries).

template <typename C>
__device__ __forceinline__ C ldt(const double2* t, int i) {
  const double2 v = __ldg(t + i);
  return cx<C>(v.x, v.y);
}

template <typename C>
__global__ void __launch_bounds__(256) k_fuse(const double2* __restrict__ t, int d, int Dfull, int4 n4,
                                              const double2* __restrict__ op, int4 perm4, C* __restrict__ T,
                                              int total) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int nn[4] = {n4.x, n4.y, n4.z, n4.w};
  const int pp[4] = {perm4.x, perm4.y, perm4.z, perm4.w};
  int ket[4], bra[4];
  int rem = idx;
#pragma unroll
  for (int q = 3; q >= 0; --q) {
    const int leg = pp[q];
    const int f2 = nn[leg] * nn[leg];
    const int f = rem % f2;
    rem /= f2;
    ket[leg] = f / nn[leg];
    bra[leg] = f % nn[leg];
  }
  const int D = Dfull;
  const int sD4 = D * D * D * D;
  const int ok = ((ket[0] * D + ket[1]) * D + ket[2]) * D + ket[3];
  const int ob = ((bra[0] * D + bra[1]) * D + bra[2]) * D + bra[3];
  if (op) {
    double2 acc = make_double2(0.0, 0.0);
    for (int s = 0; s < d; ++s) {
      const double2 tb = cconj(t[s * sD4 + ob]);
      for (int sp = 0; sp < d; ++sp) acc = cadd(acc, cmul(op[s * d + sp], cmul(t[sp * sD4 + ok], tb)));
    }
    T[idx] = cx<C>(acc.x, acc.y);
    return;
  }
  C acc = cx<C>(0.0, 0.0);
  for (int s = 0; s < d; ++s) acc = cadd(acc, cmul(ldt<C>(t, s * sD4 + ok), cconj(ldt<C>(t, s * sD4 + ob))));
  T[idx] = acc;
}

// -------------------------------------------------------------------- gemm

constexpr int GT = 32;   // output tile
constexpr int GK = 16;   // k tile

template <typename C>
__device__ __forceinline__ C load_op(const C* P, int ld, char op, int r, int c, int R, int Cc) {
  if (r >= R || c >= Cc) return cx<C>(0, 0);
  if (op == 'N') return P[(long long)r * ld + c];
  C v = P[(long long)c * ld + r];
  return op == 'C' ? cconj(v) : v;
}

// With part != null the grid's z index is a slice of K (kchunk entries,
// batch 1): each CTA writes its raw partial tile to part[z][M][N] and
// k_gemm_reduce adds the slices in order (split K for skinny products).
template <typename C>
__global__ void __launch_bounds__(256) k_gemm(char opA, char opB, int M, int N, int K, C alpha, const C* __restrict__ A,
                                              int lda, long long sA, const C* __restrict__ B, int ldb, long long sB,
                                              C beta, C* __restrict__ Cm, int ldc, long long sC, int kchunk,
                                              C* __restrict__ part) {
  __shared__ C As[GT][GK + 1];
  __shared__ C Bs[GK][GT + 1];
  const int bz = blockIdx.z;
  int kb = 0, ke = K;
  if (part) {
    kb = bz * kchunk;
    ke = min(K, kb + kchunk);
  } else {
    A += bz * sA;
    B += bz * sB;
    Cm += bz * sC;
  }
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  C acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = cx<C>(0, 0);
  // the next k tile is loaded into registers while the current one is
  // multiplied (GT * GK / 256 = 2 entries of A and 2 of B a thread)
  constexpr int kPer = GT * GK / 256;
  C pa[kPer], pb[kPer];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = threadIdx.x + 256 * u;
      pa[u] = load_op(A, lda, opA, row0 + e / GK, k0 + e % GK, M, ke);
      pb[u] = load_op(B, ldb, opB, k0 + e / GT, col0 + e % GT, ke, N);
    }
  };
  if (kb < ke) fetch(kb);
  for (int k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = threadIdx.x + 256 * u;
      As[e / GK][e % GK] = pa[u];
      Bs[e / GT][e % GT] = pb[u];
    }
    __syncthreads();
    if (k0 + GK < ke) fetch(k0 + GK);
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      C a0 = As[ty][kk], a1 = As[ty + 16][kk];
      C b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = cadd(acc[0][0], cmul(a0, b0));
      acc[0][1] = cadd(acc[0][1], cmul(a0, b1));
      acc[1][0] = cadd(acc[1][0], cmul(a1, b0));
      acc[1][1] = cadd(acc[1][1], cmul(a1, b1));
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < M && c < N) {
        if (part) {
          part[((long long)bz * M + r) * N + c] = acc[i][j];
          continue;
        }
        C v = cmul(alpha, acc[i][j]);
        if (beta.x != 0 || beta.y != 0) v = cadd(v, cmul(beta, Cm[(long long)r * ldc + c]));
        Cm[(long long)r * ldc + c] = v;
      }
    }
}

template <typename C>
__global__ void k_gemm_reduce(const C* __restrict__ part, int S, int M, int N, C alpha, C beta, C* __restrict__ Cm,
                              int ldc) {
  const long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    C v = part[e];
    for (int z = 1; z < S; ++z) v = cadd(v, part[(long long)z * tot + e]);
    const int r = (int)(e / N), c = (int)(e % N);
    v = cmul(alpha, v);
    if (beta.x != 0 || beta.y != 0) v = cadd(v, cmul(beta, Cm[(long long)r * ldc + c]));
    Cm[(long long)r * ldc + c] = v;
  }
}

// ---------------------------------------------------------------------- QR
// Householder with real diagonal of R (H = I - tau v v^H, v_j = 1).  One CTA
// of 256 threads; A (m x n, row-major, ld = n) is overwritten by R and the
// reflectors.  Lanes map to consecutive columns and warps to row groups, so
// every row access of the trailing update is a coalesced 32-column stripe.

template <typename C>
__device__ void cta_householder(C* A, int m, int n, C* tau, double* sh) {
  const int k = m < n ? m : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double s_tau[2], s_scale[2];
  __shared__ C s_w[8][33];
  for (int j = 0; j < k; ++j) {
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) part += cabs2d(A[(long long)i * n + j]);
    double xn2 = block_sum(part, sh);
    if (threadIdx.x == 0) {
      double2 alpha = c128(A[(long long)j * n + j]);
      if (xn2 == 0.0 && alpha.y == 0.0) {
        s_tau[0] = s_tau[1] = 0.0;
        s_scale[0] = s_scale[1] = 0.0;
      } else {
        double beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
        s_tau[0] = (beta - alpha.x) / beta;
        s_tau[1] = -alpha.y / beta;
        double dx = alpha.x - beta, dy = alpha.y, dd = dx * dx + dy * dy;
        s_scale[0] = dx / dd;
        s_scale[1] = -dy / dd;
        A[(long long)j * n + j] = cx<C>(beta, 0.0);
      }
      tau[j] = cx<C>(s_tau[0], s_tau[1]);
    }
    __syncthreads();
    const C tj = cx<C>(s_tau[0], s_tau[1]), sc = cx<C>(s_scale[0], s_scale[1]);
    if (tj.x == 0 && tj.y == 0) { __syncthreads(); continue; }
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[(long long)i * n + j] = cmul(A[(long long)i * n + j], sc);
    __syncthreads();
    // A[j:, c] -= conj(tau) v (v^H A[j:, c]) for c > j, 32 columns at a time
    const C ctau = cconj(tj);
    for (int cb = j + 1; cb < n; cb += 32) {
      const int c = cb + lane;
      C acc = cx<C>(0, 0);
      if (c < n)
        for (int i = j + wid; i < m; i += nw) {
          C v = (i == j) ? cx<C>(1, 0) : A[(long long)i * n + j];
          acc = cadd(acc, cmulc(v, A[(long long)i * n + c]));
        }
      s_w[wid][lane] = acc;
      __syncthreads();
      if (wid == 0) {
        C t = s_w[0][lane];
        for (int g = 1; g < nw; ++g) t = cadd(t, s_w[g][lane]);
        s_w[0][lane] = cmul(ctau, t);
      }
      __syncthreads();
      const C f = s_w[0][lane];
      if (c < n)
        for (int i = j + wid; i < m; i += nw) {
          C v = (i == j) ? cx<C>(1, 0) : A[(long long)i * n + j];
          A[(long long)i * n + c] = csub(A[(long long)i * n + c], cmul(v, f));
        }
      __syncthreads();
    }
  }
}

// Q (m x k, row-major) from the reflectors stored in A (one CTA of 256 threads).
template <typename C>
__device__ void cta_form_q(const C* A, int m, int n, const C* tau, C* Q) {
  const int k = m < n ? m : n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ C s_w[8][33];
  for (long long e = threadIdx.x; e < (long long)m * k; e += blockDim.x) {
    int i = (int)(e / k), c = (int)(e % k);
    Q[e] = cx<C>(i == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const C tj = tau[j];
    if (tj.x == 0 && tj.y == 0) continue;
    for (int cb = j; cb < k; cb += 32) {
      const int c = cb + lane;
      C acc = cx<C>(0, 0);
      if (c < k)
        for (int i = j + wid; i < m; i += nw) {
          C v = (i == j) ? cx<C>(1, 0) : A[(long long)i * n + j];
          acc = cadd(acc, cmulc(v, Q[(long long)i * k + c]));
        }
      s_w[wid][lane] = acc;
      __syncthreads();
      if (wid == 0) {
        C t = s_w[0][lane];
        for (int g = 1; g < nw; ++g) t = cadd(t, s_w[g][lane]);
        s_w[0][lane] = cmul(tj, t);
      }
      __syncthreads();
      const C f = s_w[0][lane];
      if (c < k)
        for (int i = j + wid; i < m; i += nw) {
          C v = (i == j) ? cx<C>(1, 0) : A[(long long)i * n + j];
          Q[(long long)i * k + c] = csub(Q[(long long)i * k + c], cmul(v, f));
        }
      __syncthreads();
    }
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_qr(C* A, int m, int n, C* Q, C* Rm, C* tau) {
  __shared__ double sh[40];
  cta_householder(A, m, n, tau, sh);
  const int k = m < n ? m : n;
  if (Rm)
    for (long long e = threadIdx.x; e < (long long)k * n; e += blockDim.x) {
      int i = (int)(e / n), c = (int)(e % n);
      Rm[e] = (c >= i) ? A[(long long)i * n + c] : cx<C>(0, 0);
    }
  __syncthreads();
  cta_form_q(A, m, n, tau, Q);
}

// dynamic shared memory of the staged kernels: the 227 KB opt-in per CTA less
// a margin for their static shared arrays
constexpr int kSmemMax = 211 * 1024;

// QR with the matrix staged in shared memory, column-major with a padded
// column stride (m + 1), one warp per column (column c belongs to warp
// c % 32, lanes run over rows).  Householder step j: every warp applies
// H_j to its columns right of j, reading the unscaled column j; the owner
// of column j + 1 then forms the next reflector's parameters, and the owner
// of column j writes v_j and beta_j once nobody reads column j any more;
// one barrier per step.  Q is formed in place backwards, the next reflector
// prefetched into a double buffer, again one barrier per step.  Same
// convention as cta_householder: R has a real diagonal beta_j,
// Q = H_0 ... H_{k-1}, H = I - tau v v^H.
template <typename C>
struct TsqrSmem {
  static size_t bytes(int m, int n) {   // column-major (m + 1) x n or row-major m x (n + 1) panel
    const int k = m < n ? m : n;
    return sizeof(C) * ((size_t)m * n + (size_t)(m > n ? m : n) + 2 * (size_t)m + 3 * (size_t)k + 8);
  }
};

template <typename C>
__device__ void tsqr_params(const C* col, int j, int m, C* s_tau, C* s_sc, C* s_beta) {
  // reflector of column j (rows j..m-1); computed by one warp in the
  // element's real type, with the column scaled by its largest magnitude
  // first so that tiny columns neither underflow nor divide by zero
  using R = typename RealOf<C>::T;
  const int lane = threadIdx.x & 31;
  const C alpha = col[j];
  R amax = fmax(fabs(alpha.x), fabs(alpha.y));
  for (int r = j + 1 + lane; r < m; r += 32) amax = fmax(amax, fmax(fabs(col[r].x), fabs(col[r].y)));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const R sa = (amax > (R)0 && isfinite(amax)) ? (R)1 / amax : (R)0;
  R xn2 = 0;
  for (int r = j + 1 + lane; r < m; r += 32) xn2 += cabs2(cscale(col[r], sa));
  xn2 = warp_sum(xn2);
  if (lane == 0) {
    C tau = cx<C>(0, 0), sc = cx<C>(0, 0), beta = alpha;
    if (sa > (R)0 && !(xn2 == (R)0 && alpha.y == (R)0)) {
      const R ax = alpha.x * sa, ay = alpha.y * sa;          // scaled, |.| <= 1
      const R bs = -copysign(sqrt(ax * ax + ay * ay + xn2), ax);
      const R dx = ax - bs, dy = ay, dd = dx * dx + dy * dy;
      const R ib = (R)1 / bs, idd = sa / dd;                 // 1 / (alpha - beta) = sa conj(d') / |d'|^2
      tau = cx<C>((bs - ax) * ib, -ay * ib);
      sc = cx<C>(dx * idd, -dy * idd);
      beta = cx<C>(bs * amax, 0.0);
      if (!(isfinite(tau.x) && isfinite(tau.y) && isfinite(sc.x) && isfinite(sc.y) && isfinite(beta.x))) {
        tau = cx<C>(0, 0);                                     // leave the column as it is
        sc = cx<C>(0, 0);
        beta = alpha;
      }
    }
    s_tau[j] = tau;
    s_sc[j] = sc;
    s_beta[j] = beta;
  }
}

template <typename C>
__global__ void __launch_bounds__(1024) k_tsqr_smem(const C* __restrict__ Ag, int m_all, int n, C* __restrict__ Q,
                                                    C* __restrict__ Rm, int rb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int row0 = blockIdx.x * rb;
  const int m = min(rb, m_all - row0);
  Ag += (size_t)row0 * n;
  if (gridDim.x > 1) Rm += (size_t)blockIdx.x * n * n;
  const int k = m < n ? m : n;
  const int ld = m + 1;
  C* A = (C*)smem_raw;                       // column c at A + c * ld
  C* vbuf = A + (size_t)ld * n;              // 2 x m
  C* s_tau = vbuf + 2 * (size_t)m;
  C* s_sc = s_tau + k;
  C* s_beta = s_sc + k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long long e = threadIdx.x; e < (long long)m * n; e += blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    A[(size_t)c * ld + r] = Ag[e];
  }
  __syncthreads();
  if (warp == 0 && k > 0) tsqr_params(A, 0, m, s_tau, s_sc, s_beta);
  __syncthreads();
  // ---- factorisation
  for (int j = 0; j < k; ++j) {
    const C* cj = A + (size_t)j * ld;
    const C tj = s_tau[j], sc = s_sc[j];
    const C ctau = cconj(tj);
    if (j > 0 && warp == (j - 1) % nw) {     // finalise column j - 1 (no longer read)
      C* cp = A + (size_t)(j - 1) * ld;
      const C scp = s_sc[j - 1];
      for (int r = j + lane; r < m; r += 32) cp[r] = cmul(cp[r], scp);
      if (lane == 0) cp[j - 1] = s_beta[j - 1];
    }
    if (!(tj.x == 0 && tj.y == 0)) {
      for (int c = j + 1 + ((warp - (j + 1)) % nw + nw) % nw; c < n; c += nw) {
        C* cc = A + (size_t)c * ld;
        C acc = cx<C>(0, 0);
        for (int r = j + 1 + lane; r < m; r += 32) acc = cadd(acc, cmulc(cj[r], cc[r]));
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        // v^H a = a_j + conj(sc) sum conj(x_r) a_r
        const C dot = cadd(cc[j], cmulc(sc, acc));
        const C f = cmul(ctau, dot);       // a -= conj(tau) v (v^H a)
        const C fs = cmul(f, sc);
        for (int r = j + 1 + lane; r < m; r += 32) cc[r] = csub(cc[r], cmul(cj[r], fs));
        if (lane == 0) cc[j] = csub(cc[j], f);
      }
    }
    __syncwarp();
    if (j + 1 < k && warp == (j + 1) % nw) tsqr_params(A + (size_t)(j + 1) * ld, j + 1, m, s_tau, s_sc, s_beta);
    __syncthreads();
  }
  if (k > 0 && warp == (k - 1) % nw) {
    C* cp = A + (size_t)(k - 1) * ld;
    const C scp = s_sc[k - 1];
    for (int r = k + lane; r < m; r += 32) cp[r] = cmul(cp[r], scp);
    if (lane == 0) cp[k - 1] = s_beta[k - 1];
  }
  __syncthreads();
  if (Rm) {
    const int krows = gridDim.x > 1 ? n : k;
    for (long long e = threadIdx.x; e < (long long)krows * n; e += blockDim.x) {
      const int i = (int)(e / n), c = (int)(e % n);
      Rm[e] = (i < k && c >= i) ? A[(size_t)c * ld + i] : cx<C>(0, 0);
    }
  }
  if (!Q) return;
  // ---- Q = H_0 ... H_{k-1} [I; 0], backwards, in place over columns 0..k-1
  if (warp == (k - 1) % nw && k > 0) {
    const C* cp = A + (size_t)(k - 1) * ld;
    for (int r = k - 1 + lane; r < m; r += 32) vbuf[((k - 1) & 1) * m + r] = (r == k - 1) ? cx<C>(1, 0) : cp[r];
  }
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const C* v = vbuf + (i & 1) * m;
    const C ti = s_tau[i];
    for (int c = i + 1 + ((warp - (i + 1)) % nw + nw) % nw; c < k; c += nw) {
      C* cc = A + (size_t)c * ld;
      C acc = cx<C>(0, 0);
      for (int r = i + lane; r < m; r += 32) acc = cadd(acc, cmulc(v[r], cc[r]));
      acc.x = warp_sum(acc.x);
      acc.y = warp_sum(acc.y);
      const C f = cmul(ti, acc);
      for (int r = i + lane; r < m; r += 32) cc[r] = csub(cc[r], cmul(v[r], f));
    }
    if (warp == i % nw) {                   // column i := e_i - tau_i v_i
      C* ci = A + (size_t)i * ld;
      const C mt = cx<C>(-ti.x, -ti.y);
      for (int r = lane; r < m; r += 32) {
        C q = cx<C>(0, 0);
        if (r == i) q = cx<C>(1.0 - ti.x, -ti.y);
        else if (r > i) q = cmul(mt, v[r]);
        ci[r] = q;
      }
    }
    if (i > 0 && warp == (i - 1) % nw) {    // prefetch v_{i-1}
      const C* cp = A + (size_t)(i - 1) * ld;
      for (int r = i - 1 + lane; r < m; r += 32) vbuf[((i - 1) & 1) * m + r] = (r == i - 1) ? cx<C>(1, 0) : cp[r];
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)m * k; e += blockDim.x) {
    const int r = (int)(e / k), c = (int)(e % k);
    Q[e] = A[(size_t)c * ld + r];
  }
}


// complex64 variant of k_tsqr_smem: the panel is kept row-major with an odd
// row stride (n + 1, so that a warp reading one column down 32 rows touches
// distinct banks), global loads and stores run along rows, and the columns a
// warp works on are cached in registers: lane l holds rows l + 32 i,
// i < MAXR (m <= 32 MAXR), so every column pass issues its loads back to
// back; 16 warps.  Same steps, barriers and results as k_tsqr_smem.
template <int MAXR>
__device__ __forceinline__ void tsqr_params_reg(const float2* A, int ldr, int c, int j, int m, float2* s_tau,
                                                float2* s_sc, float2* s_beta) {
  const int lane = threadIdx.x & 31;
  float2 x[MAXR];
#pragma unroll
  for (int i = 0; i < MAXR; ++i) {
    const int r = lane + 32 * i;
    x[i] = (r > j && r < m) ? A[(size_t)r * ldr + c] : make_float2(0.f, 0.f);
  }
  const float2 alpha = A[(size_t)j * ldr + c];
  float amax = fmaxf(fabsf(alpha.x), fabsf(alpha.y));
#pragma unroll
  for (int i = 0; i < MAXR; ++i) amax = fmaxf(amax, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const float sa = (amax > 0.f && isfinite(amax)) ? 1.f / amax : 0.f;
  float xn2 = 0.f;
#pragma unroll
  for (int i = 0; i < MAXR; ++i) xn2 += (x[i].x * sa) * (x[i].x * sa) + (x[i].y * sa) * (x[i].y * sa);
  xn2 = warp_sum(xn2);
  if (lane == 0) {
    float2 tau = make_float2(0.f, 0.f), sc = make_float2(0.f, 0.f), beta = alpha;
    if (sa > 0.f && !(xn2 == 0.f && alpha.y == 0.f)) {
      const float ax = alpha.x * sa, ay = alpha.y * sa;
      const float bs = -copysignf(sqrtf(ax * ax + ay * ay + xn2), ax);
      const float dx = ax - bs, dy = ay, dd = dx * dx + dy * dy;
      const float ib = 1.f / bs, idd = sa / dd;
      tau = make_float2((bs - ax) * ib, -ay * ib);
      sc = make_float2(dx * idd, -dy * idd);
      beta = make_float2(bs * amax, 0.f);
      if (!(isfinite(tau.x) && isfinite(tau.y) && isfinite(sc.x) && isfinite(sc.y) && isfinite(beta.x))) {
        tau = make_float2(0.f, 0.f);
        sc = make_float2(0.f, 0.f);
        beta = alpha;
      }
    }
    s_tau[j] = tau;
    s_sc[j] = sc;
    s_beta[j] = beta;
  }
}

inline size_t tsqr_reg_bytes(int m, int n) {
  const int k = m < n ? m : n;
  return sizeof(float2) * ((size_t)m * (n + 1) + 2 * (size_t)m + 3 * (size_t)k + 8);
}

template <int MAXR>
__global__ void __launch_bounds__(512, 1) k_tsqr_reg(const float2* __restrict__ Ag, int m_all, int n, float2* Q,
                                                     float2* Rm, int rb) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int row0 = blockIdx.x * rb;
  const int m = min(rb, m_all - row0);
  Ag += (size_t)row0 * n;
  if (gridDim.x > 1) Rm += (size_t)blockIdx.x * n * n;
  const int k = m < n ? m : n;
  const int ldr = n + 1;
  C* A = (C*)smem_raw;                       // (r, c) at A[r * ldr + c]
  C* vbuf = A + (size_t)m * ldr;
  C* s_tau = vbuf + 2 * (size_t)m;
  C* s_sc = s_tau + k;
  C* s_beta = s_sc + k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < n; c0 += 64)
    for (int r0 = warp * 4; r0 < m; r0 += nw * 4) {
      C v[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = r0 + q, c = c0 + lane + 32 * h;
          v[q][h] = (r < m && c < n) ? Ag[(size_t)r * n + c] : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = r0 + q, c = c0 + lane + 32 * h;
          if (r < m && c < n) A[(size_t)r * ldr + c] = v[q][h];
        }
    }
  __syncthreads();
  if (warp == 0 && k > 0) tsqr_params_reg<MAXR>(A, ldr, 0, 0, m, s_tau, s_sc, s_beta);
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const C tj = s_tau[j], sc = s_sc[j];
    const C ctau = cconj(tj);
    if (j > 0 && warp == (j - 1) % nw) {     // finalise column j - 1
      const C scp = s_sc[j - 1];
      for (int r = j + lane; r < m; r += 32) A[(size_t)r * ldr + j - 1] = cmul(A[(size_t)r * ldr + j - 1], scp);
      if (lane == 0) A[(size_t)(j - 1) * ldr + j - 1] = s_beta[j - 1];
    }
    const int c0 = j + 1 + ((warp - (j + 1)) % nw + nw) % nw;
    if (!(tj.x == 0.f && tj.y == 0.f) && c0 < n) {
      C xj[MAXR];
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const int r = lane + 32 * i;
        xj[i] = (r > j && r < m) ? A[(size_t)r * ldr + j] : make_float2(0.f, 0.f);
      }
      for (int c = c0; c < n; c += nw) {
        C y[MAXR];
#pragma unroll
        for (int i = 0; i < MAXR; ++i) {
          const int r = lane + 32 * i;
          y[i] = (r > j && r < m) ? A[(size_t)r * ldr + c] : make_float2(0.f, 0.f);
        }
        C a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < MAXR; i += 2) {
          a0 = cadd(a0, cmulc(xj[i], y[i]));
          if (i + 1 < MAXR) a1 = cadd(a1, cmulc(xj[i + 1], y[i + 1]));
        }
        C acc = cadd(a0, a1);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        const C ajc = A[(size_t)j * ldr + c];
        const C dot = cadd(ajc, cmulc(sc, acc));
        const C f = cmul(ctau, dot);
        const C fs = cmul(f, sc);
#pragma unroll
        for (int i = 0; i < MAXR; ++i) {
          const int r = lane + 32 * i;
          if (r > j && r < m) A[(size_t)r * ldr + c] = csub(y[i], cmul(xj[i], fs));
        }
        __syncwarp();
        if (lane == 0) A[(size_t)j * ldr + c] = csub(ajc, f);
      }
    }
    __syncwarp();
    if (j + 1 < k && warp == (j + 1) % nw) tsqr_params_reg<MAXR>(A, ldr, j + 1, j + 1, m, s_tau, s_sc, s_beta);
    __syncthreads();
  }
  if (k > 0 && warp == (k - 1) % nw) {
    const C scp = s_sc[k - 1];
    for (int r = k + lane; r < m; r += 32) A[(size_t)r * ldr + k - 1] = cmul(A[(size_t)r * ldr + k - 1], scp);
    if (lane == 0) A[(size_t)(k - 1) * ldr + k - 1] = s_beta[k - 1];
  }
  __syncthreads();
  if (Rm) {
    const int krows = gridDim.x > 1 ? n : k;
    for (int i = warp; i < krows; i += nw)
      for (int c = lane; c < n; c += 32)
        Rm[(size_t)i * n + c] = (i < k && c >= i) ? A[(size_t)i * ldr + c] : make_float2(0.f, 0.f);
  }
  if (!Q) return;
  if (k > 0 && warp == (k - 1) % nw)
    for (int r = k - 1 + lane; r < m; r += 32)
      vbuf[((k - 1) & 1) * m + r] = (r == k - 1) ? make_float2(1.f, 0.f) : A[(size_t)r * ldr + k - 1];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const C* v = vbuf + (i & 1) * m;
    const C ti = s_tau[i];
    const int c0 = i + 1 + ((warp - (i + 1)) % nw + nw) % nw;
    const bool own_i = warp == i % nw;
    if (c0 < k || own_i) {
      C vv[MAXR];
#pragma unroll
      for (int q = 0; q < MAXR; ++q) {
        const int r = lane + 32 * q;
        vv[q] = (r >= i && r < m) ? v[r] : make_float2(0.f, 0.f);
      }
      for (int c = c0; c < k; c += nw) {
        C y[MAXR];
#pragma unroll
        for (int q = 0; q < MAXR; ++q) {
          const int r = lane + 32 * q;
          y[q] = (r >= i && r < m) ? A[(size_t)r * ldr + c] : make_float2(0.f, 0.f);
        }
        C a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < MAXR; q += 2) {
          a0 = cadd(a0, cmulc(vv[q], y[q]));
          if (q + 1 < MAXR) a1 = cadd(a1, cmulc(vv[q + 1], y[q + 1]));
        }
        C acc = cadd(a0, a1);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        const C f = cmul(ti, acc);
#pragma unroll
        for (int q = 0; q < MAXR; ++q) {
          const int r = lane + 32 * q;
          if (r >= i && r < m) A[(size_t)r * ldr + c] = csub(y[q], cmul(vv[q], f));
        }
      }
      if (own_i) {                          // column i := e_i - tau_i v_i
        const C mt = make_float2(-ti.x, -ti.y);
#pragma unroll
        for (int q = 0; q < MAXR; ++q) {
          const int r = lane + 32 * q;
          if (r < m)
            A[(size_t)r * ldr + i] =
                (r == i) ? make_float2(1.f - ti.x, -ti.y) : (r > i ? cmul(mt, vv[q]) : make_float2(0.f, 0.f));
        }
      }
    }
    if (i > 0 && warp == (i - 1) % nw)
      for (int r = i - 1 + lane; r < m; r += 32)
        vbuf[((i - 1) & 1) * m + r] = (r == i - 1) ? make_float2(1.f, 0.f) : A[(size_t)r * ldr + i - 1];
    __syncthreads();
  }
  for (int r = warp; r < m; r += nw)
    for (int c = lane; c < k; c += 32) Q[(size_t)r * k + c] = A[(size_t)r * ldr + c];
}

// One staged QR launch (grid = row blocks): the register-cached kernel for
// complex64 panels of at most 512 rows per block, the generic one otherwise.
template <typename C>
cudaError_t tsqr_launch(const C* Ag, int m_all, int n, C* Q, C* Rm, int rb, cudaStream_t s);

template <>
cudaError_t tsqr_launch<float2>(const float2* Ag, int m_all, int n, float2* Q, float2* Rm, int rb, cudaStream_t s) {
  const int nb = (m_all + rb - 1) / rb;
  const size_t sr = tsqr_reg_bytes(rb, n);
  if (rb <= 128 && sr <= (size_t)kSmemMax) k_tsqr_reg<4><<<nb, 512, sr, s>>>(Ag, m_all, n, Q, Rm, rb);
  else if (rb <= 256 && sr <= (size_t)kSmemMax) k_tsqr_reg<8><<<nb, 512, sr, s>>>(Ag, m_all, n, Q, Rm, rb);
  else if (rb <= 512 && sr <= (size_t)kSmemMax) k_tsqr_reg<16><<<nb, 512, sr, s>>>(Ag, m_all, n, Q, Rm, rb);
  else k_tsqr_smem<float2><<<nb, 1024, TsqrSmem<float2>::bytes(rb, n), s>>>(Ag, m_all, n, Q, Rm, rb);
  return cudaGetLastError();
}

template <>
cudaError_t tsqr_launch<double2>(const double2* Ag, int m_all, int n, double2* Q, double2* Rm, int rb,
                                 cudaStream_t s) {
  const int nb = (m_all + rb - 1) / rb;
  k_tsqr_smem<double2><<<nb, 1024, TsqrSmem<double2>::bytes(rb, n), s>>>(Ag, m_all, n, Q, Rm, rb);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- K3 Jacobi

template <typename C>
struct SvdWork {
  C* G;
  C* WH;
  double* sigma;
  int* idx;
  int* counters;   // [0..1] rotations per sweep, [2] sweeps, [3] rotations in total
  double* zn2;     // ||Z||_F^2
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename C>
__host__ __device__ inline SvdWork<C> carve(void* work, int M, int N) {
  char* p = (char*)work;
  SvdWork<C> w;
  w.G = (C*)p; p += align256(sizeof(C) * (size_t)M * N);
  w.WH = (C*)p; p += align256(sizeof(C) * (size_t)M * M);
  w.sigma = (double*)p; p += align256(sizeof(double) * (size_t)M);
  w.idx = (int*)p; p += align256(sizeof(int) * (size_t)M);
  w.counters = (int*)p;
  w.zn2 = (double*)(p + 32);
  return w;
}

template <typename C>
size_t jacobi_bytes(int M, int N) {
  return align256(sizeof(C) * (size_t)M * N) + align256(sizeof(C) * (size_t)M * M) + align256(sizeof(double) * M) +
         align256(sizeof(int) * M) + 256;
}
template <typename C> static bool jacobi_reduce_fits(int M, int N);
template <typename C> static size_t jacobi_reduce_bytes(int M, int N);
// scratch of jacobi_svd, including the QR reduction of long matrices
template <typename C>
size_t jacobi_svd_bytes(int M, int N) {
  return jacobi_bytes<C>(M, N) + (jacobi_reduce_fits<C>(M, N) ? jacobi_reduce_bytes<C>(M, N) : 0);
}

// Copies Z (or Z^H) into G, sets WH = I and accumulates ||Z||^2 into *zn2;
// the counters and *zn2 are zeroed by the caller before the launch.
template <typename C>
__global__ void k_svd_init(const C* __restrict__ Z, int m, int n, SvdWork<C> w) {
  __shared__ double sh[40];
  const int M = m <= n ? m : n, N = m <= n ? n : m;
  long long tot = (long long)M * N, totw = (long long)M * M;
  double part = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot + totw;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < tot) {
      int a = (int)(e / N), c = (int)(e % N);
      C v = (m <= n) ? Z[(long long)a * n + c] : cconj(Z[(long long)c * n + a]);
      w.G[e] = v;
      part += cabs2d(v);
    } else {
      long long f = e - tot;
      int a = (int)(f / M), c = (int)(f % M);
      w.WH[f] = cx<C>(a == c ? 1.0 : 0.0, 0.0);
    }
  }
  double bs = block_sum(part, sh);
  if (threadIdx.x == 0) atomicAdd(w.zn2, bs);
}

template <typename C>
__device__ __forceinline__ C ldcg(const C* p);
template <> __device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }
template <typename C>
__device__ __forceinline__ void stcg(C* p, C v);
template <> __device__ __forceinline__ void stcg(double2* p, double2 v) { __stcg(p, v); }
template <> __device__ __forceinline__ void stcg(float2* p, float2 v) { __stcg(p, v); }
// rows in global memory bypass L1 (other CTAs of the cluster rotate them);
// rows in shared memory are plain accesses
template <bool kGlobal, typename C> __device__ __forceinline__ C ldrow(const C* p) { return kGlobal ? ldcg(p) : *p; }
template <bool kGlobal, typename C> __device__ __forceinline__ void strow(C* p, C v) {
  if (kGlobal) stcg(p, v);
  else *p = v;
}

// Rotate rows a, b of G (length N) and of WH (length M) so that they become
// orthogonal.  Warp-cooperative (all lanes take the same decision: the xor
// butterfly leaves bitwise identical sums in every lane); returns 1 when a
// rotation was applied.
template <bool kGlobal, typename C, bool kGlobalW = kGlobal>
__device__ int rotate_pair(C* ra, C* rb, int N, C* wa, C* wb, int M, int lane, double tol,
                           typename RealOf<C>::T floor) {
  using R = typename RealOf<C>::T;
  R al = 0, be = 0, gx = 0, gy = 0;
  for (int c = lane; c < N; c += 32) {
    C x = ldrow<kGlobal>(ra + c), y = ldrow<kGlobal>(rb + c);
    al += cabs2(x);
    be += cabs2(y);
    gx += x.x * y.x + x.y * y.y;      // x * conj(y)
    gy += x.y * y.x - x.x * y.y;
  }
  al = warp_sum(al);
  be = warp_sum(be);
  gx = warp_sum(gx);
  gy = warp_sum(gy);
  R g = sqrt(gx * gx + gy * gy);
  if (g == 0 || g <= (R)tol * sqrt(al) * sqrt(be)) return 0;
  // a row below eps ||Z|| carries nothing at working precision; orthogonalising
  // it (in subnormal arithmetic, at worst) would never meet the test above
  if (fmin(al, be) <= floor) return 0;
  // rows whose norms differ by more than 1e30 (1e15 in complex64) do not
  // affect each other at working precision; rotating them only churns
  // rounding noise (and never meets the relative test once a norm is subnormal)
  const R far = sizeof(R) == 8 ? (R)1e-60 : (R)1e-30;
  if (fmin(al, be) <= far * fmax(al, be)) return 0;
  C e = cx<C>(gx / g, gy / g);
  R zeta = (be - al) / (2 * g);
  R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
  R cs = (R)1 / sqrt((R)1 + t * t), sn = cs * t;
  for (int c = lane; c < N; c += 32) {
    C x = ldrow<kGlobal>(ra + c), y = ldrow<kGlobal>(rb + c);
    C ey = cmul(e, y);
    strow<kGlobal>(ra + c, csub(cscale(x, cs), cscale(ey, sn)));
    strow<kGlobal>(rb + c, cadd(cscale(x, sn), cscale(ey, cs)));
  }
  for (int c = lane; c < M; c += 32) {
    C x = ldrow<kGlobalW>(wa + c), y = ldrow<kGlobalW>(wb + c);
    C ey = cmul(e, y);
    strow<kGlobalW>(wa + c, csub(cscale(x, cs), cscale(ey, sn)));
    strow<kGlobalW>(wb + c, cadd(cscale(x, sn), cscale(ey, cs)));
  }
  return 1;
}

// The same rotation by a half warp (16 lanes: lane l of the half handles
// entries l, l + 16, ...): two pairs a warp.  Both halves always run the
// sums (an invalid pair on zeros), so the shuffles see the whole warp.
template <typename C>
__device__ int rotate_pair_half(C* ra, C* rb, int N, C* wa, C* wb, int M, int hl, bool valid, double tol,
                                typename RealOf<C>::T floor) {
  using R = typename RealOf<C>::T;
  R al = 0, be = 0, gx = 0, gy = 0;
  if (valid)
    for (int c = hl; c < N; c += 16) {
      const C x = ra[c], y = rb[c];
      al += cabs2(x);
      be += cabs2(y);
      gx += x.x * y.x + x.y * y.y;
      gy += x.y * y.x - x.x * y.y;
    }
  for (int o = 8; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
  }
  if (!valid) return 0;
  R g = sqrt(gx * gx + gy * gy);
  if (g == 0 || g <= (R)tol * sqrt(al) * sqrt(be)) return 0;
  if (fmin(al, be) <= floor) return 0;
  const R far = sizeof(R) == 8 ? (R)1e-60 : (R)1e-30;
  if (fmin(al, be) <= far * fmax(al, be)) return 0;
  C e = cx<C>(gx / g, gy / g);
  R zeta = (be - al) / (2 * g);
  R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
  R cs = (R)1 / sqrt((R)1 + t * t), sn = cs * t;
  for (int c = hl; c < N; c += 16) {
    const C x = ra[c], y = rb[c];
    const C ey = cmul(e, y);
    ra[c] = csub(cscale(x, cs), cscale(ey, sn));
    rb[c] = cadd(cscale(x, sn), cscale(ey, cs));
  }
  for (int c = hl; c < M; c += 16) {
    const C x = wa[c], y = wb[c];
    const C ey = cmul(e, y);
    wa[c] = csub(cscale(x, cs), cscale(ey, sn));
    wb[c] = cadd(cscale(x, sn), cscale(ey, cs));
  }
  return 1;
}

// Algorithmic flops of a one-sided Jacobi run: every sweep tests M(M-1)/2
// pairs (two squared norms and one complex inner product over N: 16 N), every
// applied rotation updates two rows of G and two of WH (18 per element pair).
__device__ __forceinline__ double jacobi_flops(int sweeps, long long rotations, int M, int N) {
  return (double)sweeps * 0.5 * M * (M - 1) * 16.0 * N + (double)rotations * 18.0 * (N + M);
}

template <typename C>
__global__ void __launch_bounds__(256) k_jacobi(SvdWork<C> w, int M, int N, double tol, double floor_rel,
                                                int max_sweeps, int* status, double* flops) {
  using R = typename RealOf<C>::T;
  const R floor = (R)(floor_rel * *w.zn2);
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gw = crank * nw + warp, tw = csize * nw;
  const int Mp = M + (M & 1);
  const int npairs = Mp / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rot = 0;
    for (int r = 0; r < Mp - 1; ++r) {
      for (int q = gw; q < npairs; q += tw) {
        int a, b;
        if (q == 0) { a = Mp - 1; b = r; }
        else { a = (r + q) % (Mp - 1); b = (r - q + Mp - 1) % (Mp - 1); }
        if (a >= M || b >= M) continue;
        rot += rotate_pair<true>(w.G + (long long)a * N, w.G + (long long)b * N, N, w.WH + (long long)a * M,
                           w.WH + (long long)b * M, M, lane, tol, floor);
      }
      cl.sync();
    }
    if (lane == 0 && rot) atomicAdd(&w.counters[sweep & 1], rot);
    cl.sync();
    const int total = *(volatile int*)&w.counters[sweep & 1];
    if (crank == 0 && threadIdx.x == 0) {
      w.counters[(sweep + 1) & 1] = 0;
      w.counters[2] = sweep + 1;        // sweeps done
      w.counters[3] += total;           // rotations applied
    }
    cl.sync();
    if (total == 0) {
      if (flops && crank == 0 && threadIdx.x == 0) atomicAdd(flops, jacobi_flops(sweep + 1, w.counters[3], M, N));
      return;
    }
  }
  if (crank == 0 && threadIdx.x == 0) {
    *status = 1;   // sweep limit reached
    if (flops) atomicAdd(flops, jacobi_flops(max_sweeps, w.counters[3], M, N));
  }
}

// One-CTA Jacobi with G and WH resident in shared memory
// ((M*N + M*M) * sizeof(C) <= kSmemMax); same rounds, tests and counters as
// k_jacobi, __syncthreads between rounds.
template <typename C>
__global__ void __launch_bounds__(1024) k_jacobi_smem(SvdWork<C> w, int M, int N, double tol, double floor_rel,
                                                     int max_sweeps, int* status, double* flops) {
  using R = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* G = (C*)smem_raw;
  C* WH = G + (long long)M * N;
  __shared__ int s_rot;
  const R floor = (R)(floor_rel * *w.zn2);
  for (long long e = threadIdx.x; e < (long long)M * N; e += blockDim.x) G[e] = w.G[e];
  for (long long e = threadIdx.x; e < (long long)M * M; e += blockDim.x) WH[e] = w.WH[e];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int Mp = M + (M & 1);
  const int npairs = Mp / 2;
  int sweeps = 0, rot_total = 0;
  bool converged = false;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    int rot = 0;
    const bool halves = npairs > nw;     // more pairs than warps: a pair per half warp
    for (int r = 0; r < Mp - 1; ++r) {
      if (halves) {
        const int hl = lane & 15, hw = 2 * warp + (lane >> 4);
        for (int q0 = 2 * warp; q0 < npairs; q0 += 2 * nw) {
          const int q = hw + (q0 - 2 * warp);   // this half's pair
          int a = 0, b = 0;
          if (q < npairs) {
            if (q == 0) { a = Mp - 1; b = r; }
            else { a = (r + q) % (Mp - 1); b = (r - q + Mp - 1) % (Mp - 1); }
          }
          const bool valid = q < npairs && a < M && b < M;
          const int aa = valid ? a : 0, bb = valid ? b : 0;
          rot += rotate_pair_half(G + (long long)aa * N, G + (long long)bb * N, N, WH + (long long)aa * M,
                                  WH + (long long)bb * M, M, hl, valid, tol, floor);
        }
      } else {
        for (int q = warp; q < npairs; q += nw) {
          int a, b;
          if (q == 0) { a = Mp - 1; b = r; }
          else { a = (r + q) % (Mp - 1); b = (r - q + Mp - 1) % (Mp - 1); }
          if (a >= M || b >= M) continue;
          rot += rotate_pair<false>(G + (long long)a * N, G + (long long)b * N, N, WH + (long long)a * M,
                               WH + (long long)b * M, M, lane, tol, floor);
        }
      }
      __syncthreads();
    }
    if ((halves ? (lane & 15) : lane) == 0 && rot) atomicAdd(&s_rot, rot);
    __syncthreads();
    const int total = s_rot;
    ++sweeps;
    rot_total += total;
    __syncthreads();
    if (total == 0) { converged = true; break; }
  }
  for (long long e = threadIdx.x; e < (long long)M * N; e += blockDim.x) w.G[e] = G[e];
  for (long long e = threadIdx.x; e < (long long)M * M; e += blockDim.x) w.WH[e] = WH[e];
  if (threadIdx.x == 0) {
    w.counters[2] = sweeps;
    w.counters[3] = rot_total;
    if (!converged) *status = 1;
    if (flops) atomicAdd(flops, jacobi_flops(sweeps, rot_total, M, N));
  }
}

template <typename C>
__global__ void k_row_norms(SvdWork<C> w, int M, int N) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= M) return;
  double s = 0.0;
  for (int c = lane; c < N; c += 32) s += cabs2d(w.G[(long long)row * N + c]);
  s = warp_sum(s);
  if (lane == 0) w.sigma[row] = sqrt(s);
}

template <typename C>
__global__ void k_select(SvdWork<C> w, int M, int k) {
  // a total order (non-finite norms rank last), so ranks 0..M-1 are a permutation
  for (int a = threadIdx.x; a < M; a += blockDim.x) {
    double sa = w.sigma[a];
    if (!(sa >= 0.0) || !isfinite(sa)) sa = -1.0;
    int rank = 0;
    for (int b = 0; b < M; ++b) {
      double sb = w.sigma[b];
      if (!(sb >= 0.0) || !isfinite(sb)) sb = -1.0;
      rank += (sb > sa) || (sb == sa && b < a);
    }
    if (rank < k) w.idx[rank] = a;
  }
}

template <typename C>
__global__ void k_svd_out(SvdWork<C> w, int m, int n, int k, double floor_rel, C* __restrict__ U,
                          C* __restrict__ Rem) {
  const double smin = sqrt(floor_rel * *w.zn2);
  const int M = m <= n ? m : n, N = m <= n ? n : m;
  long long totU = (long long)m * k, totR = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totU + totR;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < totU) {
      int i = (int)(e / k), r = (int)(e % k);
      int a = min(max(w.idx[r], 0), M - 1);
      if (m <= n) {
        U[e] = cconj(w.WH[(long long)a * M + i]);
      } else {
        double s = w.sigma[a];
        U[e] = (s > smin && s > 0.0) ? cscale(cconj(w.G[(long long)a * N + i]), 1.0 / s) : cx<C>(0, 0);
      }
    } else {
      long long f = e - totU;
      int r = (int)(f / n), c = (int)(f % n);
      int a = min(max(w.idx[r], 0), M - 1);
      if (m <= n) Rem[f] = w.G[(long long)a * N + c];
      else Rem[f] = cscale(w.WH[(long long)a * M + c], w.sigma[a]);
    }
  }
}

// Rows below sqrt(floor_rel) ||Z|| are left unrotated (eps^2 of the type).
template <typename C> constexpr double floor_rel_of() { return sizeof(typename RealOf<C>::T) == 8 ? 1e-32 : 1e-14; }

// Large dynamic shared memory is opt-in, once per kernel and device.
template <auto kKernel>
cudaError_t smem_optin() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kKernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

// Jacobi on the M x N rows of w: in shared memory when G and WH fit (one CTA,
// one warp per pair), else on a cluster of up to 8 CTAs.
template <typename C>
cudaError_t launch_jacobi(SvdWork<C> w, int M, int N, double tol, int max_sweeps, int* status, cudaStream_t s) {
  KTimerScope timer(KC_JACOBI, s, 0.0);
  double* flops = ktimer_device_flops(KC_JACOBI);
  const size_t jsm = sizeof(C) * ((size_t)M * N + (size_t)M * M);
  if (jsm <= (size_t)kSmemMax) {
    cudaError_t e = smem_optin<k_jacobi_smem<C>>();
    if (e != cudaSuccess) return e;
    const int threads = std::min(1024, 32 * std::max(1, (M + 1) / 2));
    k_jacobi_smem<C><<<1, threads, jsm, s>>>(w, M, N, tol, floor_rel_of<C>(), max_sweeps, status, flops);
    return cudaGetLastError();
  }
  int cs = (M / 2 + 15) / 16;   // about two pairs per warp per round
  if (cs < 1) cs = 1;
  if (cs > 8) cs = 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_jacobi<C>, w, M, N, tol, floor_rel_of<C>(), max_sweeps, status, flops);
}

// G (M x N rows of Z or Z^H) too long for shared memory but with an M x M
// square that fits: G^H = Q_T R_T (panel QR, N x M), so G = L Q_T^H with
// L = R_T^H; the Jacobi rotates L into WH L (same singular values and WH),
// and the rotated rows of G are (WH L) Q_T^H.  Scratch in the G area of w.
template <typename C>
static bool jacobi_reduce_fits(int M, int N) {
  return sizeof(C) * ((size_t)M * N + (size_t)M * M) > (size_t)kSmemMax &&
         2 * sizeof(C) * (size_t)M * M <= (size_t)kSmemMax && N >= 2 * M && panel_cluster(N, M, sizeof(C)) > 0;
}

// extra scratch of the reduction: G^H (N x M), Q_T (N x M), L and WH L (M x M)
template <typename C>
static size_t jacobi_reduce_bytes(int M, int N) {
  return 2 * align256(sizeof(C) * (size_t)N * M) + 2 * align256(sizeof(C) * (size_t)M * M);
}

template <typename C>
cudaError_t jacobi_svd(const C* Z, int m, int n, int chi, C* U, C* Rem, void* work, int* status, cudaStream_t s,
                       double tol, int max_sweeps) {
  const int M = m < n ? m : n, N = m < n ? n : m;
  const int k = chi < M ? chi : M;
  SvdWork<C> w = carve<C>(work, M, N);
  cudaError_t e0 = cudaMemsetAsync(w.counters, 0, 64, s);
  if (e0 != cudaSuccess) return e0;
  k_svd_init<C><<<grid_for((long long)M * N + (long long)M * M, 256), 256, 0, s>>>(Z, m, n, w);
  cudaError_t e;
  if (jacobi_reduce_fits<C>(M, N)) {
    char* p = (char*)work + jacobi_bytes<C>(M, N);
    C* GH = (C*)p; p += align256(sizeof(C) * (size_t)N * M);
    C* QT = (C*)p; p += align256(sizeof(C) * (size_t)N * M);
    C* Lm = (C*)p; p += align256(sizeof(C) * (size_t)M * M);
    C* LR = (C*)p;
    if ((e = launch_conj_transpose(w.G, M, N, GH, s)) != cudaSuccess) return e;
    if ((e = launch_panel_qr(GH, N, M, QT, LR, 1, 0, s)) != cudaSuccess) return e;      // R_T into LR
    if ((e = launch_conj_transpose(LR, M, M, Lm, s)) != cudaSuccess) return e;          // L = R_T^H
    // the M x M problem in its own SvdWork view (WH = I there), same counters
    SvdWork<C> ws = carve<C>(LR, M, M);
    ws.counters = w.counters;
    ws.zn2 = w.zn2;
    ws.sigma = w.sigma;
    ws.idx = w.idx;
    ws.WH = w.WH;
    ws.G = LR;
    if ((e = cudaMemcpyAsync(LR, Lm, sizeof(C) * (size_t)M * M, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    if ((e = launch_jacobi(ws, M, M, tol, max_sweeps, status, s)) != cudaSuccess) return e;
    // rotated rows of G: (WH L) Q_T^H (M x N)
    if ((e = launch_zgemm('N', 'C', M, N, M, cx<C>(1, 0), LR, M, 0, QT, M, 0, cx<C>(0, 0), w.G, N, 0, 1, s)) !=
        cudaSuccess)
      return e;
  } else {
    e = launch_jacobi(w, M, N, tol, max_sweeps, status, s);
    if (e != cudaSuccess) return e;
  }
  k_row_norms<C><<<(M * 32 + 255) / 256, 256, 0, s>>>(w, M, N);
  k_select<C><<<1, 256, 0, s>>>(w, M, k);
  k_svd_out<C><<<grid_for((long long)m * k + (long long)k * n, 256), 256, 0, s>>>(w, m, n, k, floor_rel_of<C>(), U,
                                                                                 Rem);
  return cudaGetLastError();
}

// ------------------------------------------- randomised range reduction (c64)
// Z (m x n), b = min(chi + p, m, n) columns: Q0 = orth(Z Omega); q times
// W = orth(Z^H Q), Q = orth(Z W); B = Q^H Z (b x n); Jacobi on B's rows:
// B = W_B B'; U = Q W_B[:, top], Rem = B'[top, :].  Omega is a fixed
// counter-hash sign matrix (the result does not depend on it once the
// subspace has converged).

template <typename C>
__global__ void k_omega(C* O, int n, int b) {
  long long tot = (long long)n * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    unsigned long long x = (unsigned long long)e * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    x ^= x >> 31;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 33;
    O[e] = cx<C>((x & 1) ? 1.0 : -1.0, (x & 2) ? 1.0 : -1.0);
  }
}

// FP64 finish of the reduced SVD (complex64 modes).  After the complex64
// Jacobi, the rows of G' = WH L (b x b) are orthogonal to complex64 accuracy
// and idx holds the k largest.  The rows of G' and WH are promoted to
// complex128 and every pair (kept, discarded) is rotated once more in double
// arithmetic, which makes the kept rows orthogonal to the discarded ones to
// double accuracy (the rotations within either set do not change the kept
// subspace); then the row norms and the choice of the k largest rows are
// taken in double.  The FP64 units of one SM are the bottleneck, so the rows
// of G' are spread over the shared memory of a cluster of kCutCluster CTAs
// (row r on CTA r % kCutCluster) and every round's disjoint pairs over all
// their warps, with one cluster barrier per round; WH stays in global memory.
constexpr int kCutCluster = 16;   // (a non-portable cluster size, opted in)

__global__ void __launch_bounds__(1024) k_jacobi_cut64(SvdWork<float2> w, int b, int k, double2* __restrict__ G64,
                                                       double2* __restrict__ WH64, double* __restrict__ sig64,
                                                       int* __restrict__ idx64) {
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rpc = (b + cs - 1) / cs;          // rows per CTA
  double2* G = (double2*)smem_raw;            // local rows: r = cr + cs * t at G + t * b
  int* kept = (int*)(G + (size_t)rpc * b);    // k
  int* disc = kept + k;                       // b - k
  int* mark = disc + (b - k);                 // b
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < rpc * b; e += blockDim.x) {
    const int t = e / b, c = e % b, r = cr + cs * t;
    if (r < b) G[e] = c128(w.G[(size_t)r * b + c]);
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x)
    if ((e / b) % cs == cr) __stcg(WH64 + e, c128(w.WH[e]));
  for (int e = threadIdx.x; e < b; e += blockDim.x) mark[e] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < k; e += blockDim.x) {
    const int a = min(max(w.idx[e], 0), b - 1);
    kept[e] = a;
    mark[a] = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int q = 0;
    for (int a = 0; a < b; ++a)
      if (!mark[a] && q < b - k) disc[q++] = a;
    for (; q < b - k; ++q) disc[q] = -1;     // duplicate indices in idx (never expected)
  }
  cl.sync();                                  // every CTA's rows and WH rows are in place
  auto grow = [&](int r) { return cl.map_shared_rank(G, r % cs) + (size_t)(r / cs) * b; };
  const int nd = b - k;
  const double floor = 1e-32 * (double)*w.zn2;   // eps^2 of double, as in the complex128 Jacobi
  if (nd > 0 && k > 0) {
    const int nbig = k >= nd ? k : nd, nsmall = k >= nd ? nd : k;
    const int* big = k >= nd ? kept : disc;
    const int* small = k >= nd ? disc : kept;
    for (int r = 0; r < nbig; ++r) {          // round r: pairs (big[(p + r) % nbig], small[p]), disjoint
      for (int p = cr + cs * warp; p < nsmall; p += cs * nw) {   // pairs dealt round-robin over the CTAs
        const int a = big[(p + r) % nbig], c = small[p];
        if (a < 0 || c < 0) continue;
        // rows of G' in (distributed) shared memory, rows of WH in global
        // memory past L1 (other CTAs of the cluster rotate them too)
        rotate_pair<false, double2, true>(grow(a), grow(c), b, WH64 + (size_t)a * b, WH64 + (size_t)c * b, b, lane,
                                          1e-15, floor);
      }
      cl.sync();
    }
  }
  // row norms and the selection in double (CTA 0), rows written back
  for (int t = warp; t < rpc; t += nw) {
    const int row = cr + cs * t;
    if (row >= b) continue;
    double sq = 0.0;
    for (int c = lane; c < b; c += 32) sq += cabs2d(G[(size_t)t * b + c]);
    sq = warp_sum(sq);
    if (lane == 0) __stcg(sig64 + row, sqrt(sq));
  }
  for (int e = threadIdx.x; e < rpc * b; e += blockDim.x) {
    const int t = e / b, c = e % b, r = cr + cs * t;
    if (r < b) G64[(size_t)r * b + c] = G[e];
  }
  cl.sync();                                  // sig64 complete; no remote reads after this
  if (cr != 0) return;
  for (int a = threadIdx.x; a < b; a += blockDim.x) {   // total order, non-finite norms last
    double sa = __ldcg(sig64 + a);
    if (!(sa >= 0.0) || !isfinite(sa)) sa = -1.0;
    int rank = 0;
    for (int c = 0; c < b; ++c) {
      double sc = __ldcg(sig64 + c);
      if (!(sc >= 0.0) || !isfinite(sc)) sc = -1.0;
      rank += (sc > sa) || (sc == sa && c < a);
    }
    if (rank < k) idx64[rank] = a;
  }
}

// U = Q WH[top]^H (m x k) and Rem = G'[top] W^H (k x n): WH and G' of the
// reduced SVD in complex128, Q and W in the path's element type.
// (products in the element type: Q and W carry its accuracy; for complex64
// the complex128 factors are rounded once, since FP64 arithmetic here would
// cost 64x the FP32 rate and add nothing)
template <typename C>
__device__ __forceinline__ C as_elem(double2 v) { return cx<C>(v.x, v.y); }

template <typename C>
__global__ void k_rand_out64(const C* __restrict__ Q, int m, int b, const double2* __restrict__ WH64,
                             const double2* __restrict__ G64, const int* __restrict__ idx64, const C* __restrict__ W,
                             int n, int k, C* U, C* Rem) {
  long long totU = (long long)m * k, totR = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totU + totR;
       e += (long long)gridDim.x * blockDim.x) {
    C acc = cx<C>(0.0, 0.0);
    if (e < totU) {
      const int i = (int)(e / k), a = min(max(idx64[(int)(e % k)], 0), b - 1);
      for (int j = 0; j < b; ++j) acc = cadd(acc, cmul(Q[(long long)i * b + j], cconj(as_elem<C>(WH64[(long long)a * b + j]))));
      U[e] = acc;
    } else {
      const long long f = e - totU;
      const int a = min(max(idx64[(int)(f / n)], 0), b - 1), c = (int)(f % n);
      for (int j = 0; j < b; ++j) acc = cadd(acc, cmul(as_elem<C>(G64[(long long)a * b + j]), cconj(W[(long long)c * b + j])));
      Rem[f] = acc;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers

template <typename C>
static cudaError_t fuse_t(const double2* t, int d, int Dfull, const int n[4], const double2* op, const int perm[4],
                          C* T, cudaStream_t s) {
  long long total = 1;
  for (int q = 0; q < 4; ++q) total *= (long long)n[q] * n[q];
  if (total > (1LL << 30) || (long long)d * Dfull * Dfull * Dfull * Dfull > (1LL << 30)) return cudaErrorInvalidValue;
  long long blocks = (total + 255) / 256;
  k_fuse<C><<<(unsigned)blocks, 256, 0, s>>>(t, d, Dfull, make_int4(n[0], n[1], n[2], n[3]), op,
                                             make_int4(perm[0], perm[1], perm[2], perm[3]), T, (int)total);
  return cudaGetLastError();
}
cudaError_t launch_fuse(const double2* t, int d, int D, const int n[4], const double2* op, const int perm[4], double2* T,
                        cudaStream_t s) {
  return fuse_t(t, d, D, n, op, perm, T, s);
}
cudaError_t launch_fuse(const double2* t, int d, int D, const int n[4], const double2* op, const int perm[4], float2* T,
                        cudaStream_t s) {
  return fuse_t(t, d, D, n, op, perm, T, s);
}

// K slices of a skinny product (few output tiles, long K) when a scratch of
// kSplitMax x M x N entries is given
constexpr int kSplitMax = 8;
template <typename C>
static cudaError_t gemm_t(char opA, char opB, int M, int N, int K, C alpha, const C* A, int lda, long long sA,
                          const C* B, int ldb, long long sB, C beta, C* Cm, int ldc, long long sC, int batch,
                          cudaStream_t s, void* work = nullptr, size_t work_bytes = 0) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  KTimerScope timer(KC_GEMM, s, 8.0 * M * N * (double)K * batch);
  const int tiles = ((N + GT - 1) / GT) * ((M + GT - 1) / GT);
  int S = 1;
  if (batch == 1 && work && tiles < 2 * 152 && K >= 8 * GK) {
    S = std::min(kSplitMax, std::max(2, (6 * 152) / tiles));   // about six CTAs an SM
    S = std::min(S, K / (4 * GK));
    while (S > 1 && (size_t)S * M * N * sizeof(C) > work_bytes) --S;
  }
  if (S > 1) {
    const int kchunk = ((K + S - 1) / S + GK - 1) / GK * GK;
    S = (K + kchunk - 1) / kchunk;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, S);
    k_gemm<C><<<grid, 256, 0, s>>>(opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, kchunk,
                                   (C*)work);
    k_gemm_reduce<C><<<grid_for((long long)M * N, 256), 256, 0, s>>>((const C*)work, S, M, N, alpha, beta, Cm, ldc);
    return cudaGetLastError();
  }
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, batch);
  k_gemm<C><<<grid, 256, 0, s>>>(opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, 0, nullptr);
  return cudaGetLastError();
}
cudaError_t launch_zgemm(char opA, char opB, int M, int N, int K, double2 alpha, const double2* A, int lda,
                         long long sA, const double2* B, int ldb, long long sB, double2 beta, double2* C, int ldc,
                         long long sC, int batch, cudaStream_t s) {
  return gemm_t(opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, s);
}
cudaError_t launch_zgemm(char opA, char opB, int M, int N, int K, float2 alpha, const float2* A, int lda, long long sA,
                         const float2* B, int ldb, long long sB, float2 beta, float2* C, int ldc, long long sC,
                         int batch, cudaStream_t s) {
  return gemm_t(opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, s);
}

// QR of a canonical move: one CTA when the matrix fits its shared memory, a
// cluster of CTAs for tall panels, else one CTA over global memory.
template <typename C>
static cudaError_t qr_t(C* A, int m, int n, C* Q, C* R, C* tau, cudaStream_t s) {
  const size_t sm = TsqrSmem<C>::bytes(m, n);
  if (sm > (size_t)kSmemMax && m >= n && panel_cluster(m, n, sizeof(C)) > 0)
    return launch_panel_qr(A, m, n, Q, R, 1, 0, s);
  KTimerScope timer(KC_QR, s, qr_flops(m, n));
  if (sm <= (size_t)kSmemMax) {
    cudaError_t e = tsqr_launch<C>(A, m, n, Q, R, m, s);
    if (e != cudaSuccess) return e;
  } else {
    k_qr<C><<<1, 256, 0, s>>>(A, m, n, Q, R, tau);
  }
  return cudaGetLastError();
}
// R factor only (Q discarded): row blocks that fit shared memory are
// factorised independently and their R's stacked and factorised again.
// R factor of a panel too wide for the staged kernels: Householder in
// global memory over A (overwritten), the reflector scalars in shared memory.
template <typename C>
__global__ void __launch_bounds__(256) k_qr_r_global(C* A, int m, int n, C* __restrict__ Rm) {
  __shared__ double sh[40];
  __shared__ C s_tau[512];
  cta_householder(A, m, n, s_tau, sh);
  __syncthreads();
  const int k = m < n ? m : n;
  for (long long e = threadIdx.x; e < (long long)k * n; e += blockDim.x) {
    const int i = (int)(e / n), c = (int)(e % n);
    Rm[e] = (c >= i) ? A[(long long)i * n + c] : cx<C>(0, 0);
  }
}

template <typename C>
static cudaError_t qr_r_t(const C* A, int m, int n, C* R, C* scratch0, C* scratch1, cudaStream_t s) {
  KTimerScope timer(KC_QR, s, 0.5 * qr_flops(m, n));
  if (TsqrSmem<C>::bytes(m, n) <= (size_t)kSmemMax) return tsqr_launch<C>(A, m, n, nullptr, R, m, s);
  int rb = 32;
  while (TsqrSmem<C>::bytes(rb + 32, n) <= (size_t)kSmemMax) rb += 32;
  const C* src = A;
  int rows = m;
  C* bufs[2] = {scratch0, scratch1};
  int which = 0;
  cudaError_t e;
  for (int level = 0; level < 16; ++level) {
    // the stacked panel fits one CTA or one cluster: finish there
    if (TsqrSmem<C>::bytes(rows, n) <= (size_t)kSmemMax) return tsqr_launch<C>(src, rows, n, nullptr, R, rows, s);
    if (rows >= n && panel_cluster(rows, n, sizeof(C), false) > 0)
      return launch_panel_qr(src, rows, n, nullptr, R, 1, 0, s);
    if (rb <= n) break;   // stacking row blocks would not shrink the panel
    const int nb = (rows + rb - 1) / rb;
    if ((e = tsqr_launch<C>(src, rows, n, nullptr, bufs[which], rb, s)) != cudaSuccess) return e;
    src = bufs[which];
    rows = nb * n;
    which ^= 1;
  }
  // one CTA over a copy in global memory (panels wider than any staging)
  if (std::min(m, n) > 512) return cudaErrorInvalidValue;
  if ((e = cudaMemcpyAsync(scratch0, A, sizeof(C) * (size_t)m * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  k_qr_r_global<C><<<1, 256, 0, s>>>(scratch0, m, n, R);
  return cudaGetLastError();
}

cudaError_t launch_qr_r(const double2* A, int m, int n, double2* R, double2* s0, double2* s1, cudaStream_t s) {
  return qr_r_t(A, m, n, R, s0, s1, s);
}
cudaError_t launch_qr_r(const float2* A, int m, int n, float2* R, float2* s0, float2* s1, cudaStream_t s) {
  return qr_r_t(A, m, n, R, s0, s1, s);
}

cudaError_t launch_qr(double2* A, int m, int n, double2* Q, double2* R, double2* tau, cudaStream_t s) {
  return qr_t(A, m, n, Q, R, tau, s);
}
cudaError_t launch_qr(float2* A, int m, int n, float2* Q, float2* R, float2* tau, cudaStream_t s) {
  return qr_t(A, m, n, Q, R, tau, s);
}

size_t svd_work_bytes(int m, int n) {
  int M = m < n ? m : n, N = m < n ? n : m;
  return jacobi_svd_bytes<double2>(M, N);
}

cudaError_t launch_svd_trunc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work,
                             int* status, cudaStream_t s) {
  return jacobi_svd<double2>(Z, m, n, chi, U, Rem, work, status, s, 1e-14, 60);
}

// Relative orthogonality a complex64 Jacobi sweep can reach on rows of
// length N: rounding in the dot products is about sqrt(N) eps_32.
static double jacobi_tol_c64(int N) { return std::max(2e-6, 3e-7 * std::sqrt((double)N)); }

// complex64: randomised reduction when the matrix is large, else plain Jacobi
// Reduced size of the randomised truncation: b = chi + max(8, chi / 2)
// directions; matrices whose smaller side is at most max(2 b, 64) take the
// exact Jacobi path instead (returns min(m, n)), where the subspace
// iteration would save little and its accuracy depends on the spectrum.
int rand_block(int m, int n, int chi) {
  const int M = m < n ? m : n;
  const int b = chi + (chi >= 16 ? chi / 2 : 8);
  return (M <= std::max(2 * b, 64)) ? M : b;
}

// Scratch of the randomised truncation: W (n x b), Q (m x b), R_W and L
// (b x b each), the Jacobi of L in the element type, and the complex128
// reduced factor (G64, WH64: b x b; sig64, idx64: b).
template <typename C>
static size_t orth_scratch_bytes(int m, int n, int b) {
  return align256(std::max(panel_chunk_scratch_bytes(m, b, sizeof(C)), panel_chunk_scratch_bytes(n, b, sizeof(C))));
}
template <typename C>
static size_t rand_work_bytes(int m, int n, int b) {
  const size_t z = sizeof(C), zd = sizeof(double2);
  return align256(z * (size_t)n * b) + align256(z * (size_t)m * b) + 2 * align256(z * (size_t)b * b) +
         jacobi_bytes<C>(b, b) + 2 * align256(zd * (size_t)b * b) + align256(sizeof(double) * b) +
         align256(sizeof(int) * b) + 256 + orth_scratch_bytes<C>(m, n, b) +
         align256(sizeof(C) * (size_t)kSplitMax * std::max(m, n) * b);
}

// packed operands of the tensor-core range finder: Z for Z W and for Z^H Q,
// and the small operand (W or Q)
static size_t rand_tc_bytes(int m, int n, int b) {
  return tc_zpack_bytes(false, m, n) + tc_zpack_bytes(false, n, m) + tc_zpack_bytes(false, 2 * b, std::max(m, n));
}

size_t svd_work_bytes_c64(int m, int n, int chi, bool tensor_cores) {
  int M = m < n ? m : n, N = m < n ? n : m;
  const int b = rand_block(m, n, chi);
  if (b >= M) return jacobi_svd_bytes<float2>(M, N);
  return rand_work_bytes<float2>(m, n, b) + (tensor_cores ? rand_tc_bytes(m, n, b) : 0);
}

// (the exact Jacobi only runs on splits whose smaller side is at most the
// randomisation threshold, so its scratch is bounded at that size)
size_t svd_work_bound_c64(int max_min, int max_max, int chi, bool tensor_cores) {
  const int b = chi + (chi >= 16 ? chi / 2 : 8);
  const int jm = std::min(max_min, std::max(2 * b, 64));
  return std::max(rand_work_bytes<float2>(max_max, max_max, b) +
                      (tensor_cores ? rand_tc_bytes(max_max, max_max, b) : 0),
                  jacobi_bytes<float2>(jm, max_max) + jacobi_reduce_bytes<float2>(jm, max_max));
}

// complex128 (the 1e-10 parity path): b = 2 chi directions, so that the
// subspace iteration with the default six power steps reaches the exact
// truncation to rounding on the spectra of the BlockBP splits; matrices whose
// smaller side is at most max(2 b, 64) take the exact Jacobi.
int rand_block64(int m, int n, int chi) {
  const int M = m < n ? m : n;
  const int b = 2 * chi;
  return (M <= std::max(2 * b, 64)) ? M : b;
}

size_t svd_work_bytes_rand64(int m, int n, int chi) {
  int M = m < n ? m : n, N = m < n ? n : m;
  const int b = rand_block64(m, n, chi);
  if (b >= M) return jacobi_svd_bytes<double2>(M, N);
  return rand_work_bytes<double2>(m, n, b);
}

size_t svd_work_bound_rand64(int max_min, int max_max, int chi) {
  const int jm = std::min(max_min, std::max(4 * chi, 64));
  return std::max(rand_work_bytes<double2>(max_max, max_max, 2 * chi),
                  jacobi_bytes<double2>(jm, max_max) + jacobi_reduce_bytes<double2>(jm, max_max));
}

static size_t cut64_smem(int b, int k) {
  const size_t rpc = (size_t)(b + kCutCluster - 1) / kCutCluster;
  return sizeof(double2) * rpc * b + sizeof(int) * (size_t)(2 * b + 8);
}

// Orthonormalise the columns of Y (rows x b) in place; R (b x b) too when R
// is not null: one CTA when the panel fits its shared memory, a cluster of
// CTAs otherwise.
template <typename C>
static cudaError_t orth_panel(C* Y, int rows, int b, C* R, void* chunk_scratch, cudaStream_t s) {
  if (TsqrSmem<C>::bytes(rows, b) <= (size_t)kSmemMax) {
    KTimerScope timer(KC_ORTH, s, qr_flops(rows, b));
    return tsqr_launch<C>(Y, rows, b, Y, R, rows, s);
  }
  if (panel_cluster(rows, b, sizeof(C), true) == 0) return launch_panel_qr_chunked(Y, rows, b, Y, R, chunk_scratch, s);
  return launch_panel_qr(Y, rows, b, Y, R, 1, 0, s);
}

// Randomised truncated SVD of Z (m x n) with b directions and q power steps:
// Q = orth(Z Omega); q times W = orth(Z^H Q), Q = orth(Z W); then
// Z^H Q = W R_W, so that B = Q^H Z = R_W^H W^H and the SVD runs on the b x b
// factor L = R_W^H.  Its one-sided Jacobi gives G' = WH L (rows sigma_i v_i^H
// in the W basis); U = Q WH[top]^H and Rem = G'[top] W^H.  complex64: the
// Jacobi runs in complex64 and is finished in complex128 (k_jacobi_cut64);
// complex128: the Jacobi runs in complex128.
template <typename C>
static cudaError_t rand_svd(const C* Z, int m, int n, int chi, int b, C* U, C* Rem, void* work, int* status,
                            cudaStream_t s, int power_iters, double jtol, bool tensor_cores, int* tc_err) {
  const int M = m < n ? m : n;
  const int k = chi < M ? chi : M;
  const bool c64 = sizeof(C) == sizeof(float2);
  if (c64 && cut64_smem(b, k) > (size_t)kSmemMax) return cudaErrorInvalidValue;
  const size_t z = sizeof(C), zd = sizeof(double2);
  char* p = (char*)work;
  C* W = (C*)p; p += align256(z * (size_t)n * b);
  C* Q = (C*)p; p += align256(z * (size_t)m * b);
  C* Rw = (C*)p; p += align256(z * (size_t)b * b);
  C* L = (C*)p; p += align256(z * (size_t)b * b);
  void* jw = p; p += jacobi_bytes<C>(b, b);
  double2* G64 = (double2*)p; p += align256(zd * (size_t)b * b);
  double2* WH64 = (double2*)p; p += align256(zd * (size_t)b * b);
  double* sig64 = (double*)p; p += align256(sizeof(double) * b);
  int* idx64 = (int*)p; p += align256(sizeof(int) * b) + 256;
  void* chunk = p; p += orth_scratch_bytes<C>(m, n, b);
  const size_t split_bytes = align256(sizeof(C) * (size_t)kSplitMax * std::max(m, n) * b);
  void* split = p; p += split_bytes;
  const C one = cx<C>(1.0, 0.0), zero = cx<C>(0.0, 0.0);
  cudaError_t e;
  // the range-finder products Y = Z W and W = Z^H Q: SIMT GEMMs, or (complex64
  // with tensor_cores) split-TF32 tcgen05 GEMMs with Z packed once per
  // orientation
  const bool tc = tensor_cores && sizeof(C) == sizeof(float2) && tc_err;
  void* Zn = p;
  void* Zc = (char*)Zn + (tc ? tc_zpack_bytes(false, m, n) : 0);
  void* Bp = (char*)Zc + (tc ? tc_zpack_bytes(false, n, m) : 0);
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (tc) {
      if ((e = tc_zpack_a(false, 'N', m, n, Z, n, Zn, s)) != cudaSuccess) return e;
      if ((e = tc_zpack_a(false, 'C', n, m, Z, n, Zc, s)) != cudaSuccess) return e;
    }
  }
  auto z_times = [&](const C* X, C* Y) -> cudaError_t {   // Y (m x b) = Z X, X n x b
    if constexpr (sizeof(C) == sizeof(float2)) {
      if (tc) {
        cudaError_t e2 = tc_zpack_b(false, 'N', n, b, X, b, Bp, s);
        if (e2 != cudaSuccess) return e2;
        return tc_zgemm_packed(false, m, b, n, Zn, Bp, Y, b, tc_err, s);
      }
    }
    return gemm_t('N', 'N', m, b, n, one, Z, n, 0, X, b, 0, zero, Y, b, 0, 1, s, split, split_bytes);
  };
  auto zh_times = [&](const C* X, C* Y) -> cudaError_t {  // Y (n x b) = Z^H X, X m x b
    if constexpr (sizeof(C) == sizeof(float2)) {
      if (tc) {
        cudaError_t e2 = tc_zpack_b(false, 'N', m, b, X, b, Bp, s);
        if (e2 != cudaSuccess) return e2;
        return tc_zgemm_packed(false, n, b, m, Zc, Bp, Y, b, tc_err, s);
      }
    }
    return gemm_t('C', 'N', n, b, m, one, Z, n, 0, X, b, 0, zero, Y, b, 0, 1, s, split, split_bytes);
  };
  k_omega<C><<<grid_for((long long)n * b, 256), 256, 0, s>>>(W, n, b);
  if ((e = z_times(W, Q)) != cudaSuccess) return e;
  if ((e = orth_panel<C>(Q, m, b, nullptr, chunk, s)) != cudaSuccess) return e;
  for (int it = 0; it < power_iters; ++it) {
    if ((e = zh_times(Q, W)) != cudaSuccess) return e;
    if ((e = orth_panel<C>(W, n, b, nullptr, chunk, s)) != cudaSuccess) return e;
    if ((e = z_times(W, Q)) != cudaSuccess) return e;
    if ((e = orth_panel<C>(Q, m, b, nullptr, chunk, s)) != cudaSuccess) return e;
  }
  if ((e = zh_times(Q, W)) != cudaSuccess) return e;
  if ((e = orth_panel<C>(W, n, b, Rw, chunk, s)) != cudaSuccess) return e;
  if ((e = launch_conj_transpose(Rw, b, b, L, s)) != cudaSuccess) return e;
  SvdWork<C> w = carve<C>(jw, b, b);
  if ((e = cudaMemsetAsync(w.counters, 0, 64, s)) != cudaSuccess) return e;
  k_svd_init<C><<<grid_for(2LL * b * b, 256), 256, 0, s>>>(L, b, b, w);
  if ((e = launch_jacobi(w, b, b, jtol, 60, status, s)) != cudaSuccess) return e;
  k_row_norms<C><<<(b * 32 + 255) / 256, 256, 0, s>>>(w, b, b);
  k_select<C><<<1, 256, 0, s>>>(w, b, k);
  const double2* WHo;
  const double2* Go;
  const int* idxo;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if ((e = smem_optin<k_jacobi_cut64>()) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCutCluster, 1, 1);
    cfg.blockDim = dim3(std::min(1024, 32 * std::max(1, (b + 1) / 2)), 1, 1);
    cfg.dynamicSmemBytes = cut64_smem(b, k);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCutCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((e = cudaLaunchKernelEx(&cfg, k_jacobi_cut64, w, b, k, G64, WH64, sig64, idx64)) != cudaSuccess) return e;
    WHo = WH64;
    Go = G64;
    idxo = idx64;
  } else {
    WHo = w.WH;
    Go = w.G;
    idxo = w.idx;
  }
  k_rand_out64<C><<<grid_for((long long)m * k + (long long)k * n, 256), 256, 0, s>>>(Q, m, b, WHo, Go, idxo, W, n, k,
                                                                                  U, Rem);
  return cudaGetLastError();
}

cudaError_t launch_svd_trunc(const float2* Z, int m, int n, int chi, float2* U, float2* Rem, void* work, int* status,
                             cudaStream_t s, int power_iters, bool tensor_cores, int* tc_err) {
  const int M = m < n ? m : n;
  const int b = rand_block(m, n, chi);
  if (b >= M) return jacobi_svd<float2>(Z, m, n, chi, U, Rem, work, status, s, jacobi_tol_c64(std::max(m, n)), 60);
  return rand_svd<float2>(Z, m, n, chi, b, U, Rem, work, status, s, power_iters, jacobi_tol_c64(n), tensor_cores,
                          tc_err);
}

cudaError_t launch_svd_trunc_rand64(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work,
                                    int* status, cudaStream_t s, int power_iters) {
  const int M = m < n ? m : n;
  const int b = rand_block64(m, n, chi);
  if (b >= M) return jacobi_svd<double2>(Z, m, n, chi, U, Rem, work, status, s, 1e-14, 60);
  return rand_svd<double2>(Z, m, n, chi, b, U, Rem, work, status, s, power_iters, 1e-14, false, nullptr);
}

cudaError_t svd_stats(const void* work, int m, int n, int* sweeps, long long* rotations, cudaStream_t s) {
  const int M = m < n ? m : n, N = m < n ? n : m;
  SvdWork<double2> w = carve<double2>(const_cast<void*>(work), M, N);
  int c[4];
  cudaError_t e = cudaMemcpyAsync(c, w.counters, sizeof(c), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  *sweeps = c[2];
  *rotations = c[3];
  return e;
}

// --------------------------------------------------------------- normalise

namespace {
template <typename C>
__global__ void __launch_bounds__(1024) k_normalise(C* A, long long n, double* logscale) {
  __shared__ double sh[40];
  double part = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) part += cabs2d(A[e]);
  double s = block_sum(part, sh);
  double nrm = sqrt(s);
  if (nrm > 0.0) {
    double inv = 1.0 / nrm;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) A[e] = cscale(A[e], inv);
    if (threadIdx.x == 0) *logscale += log(nrm);
  } else if (threadIdx.x == 0) {
    *logscale = -INFINITY;
  }
}

// The same normalisation over many CTAs for large tensors: partial sums of
// |A|^2 into acc (zeroed before), then every CTA scales its part by
// 1 / sqrt(acc) and CTA 0 adds log sqrt(acc) to the log-scale.
template <typename C>
__global__ void __launch_bounds__(256) k_norm_sum(const C* __restrict__ A, long long n, double* acc) {
  __shared__ double sh[40];
  double part = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    part += cabs2d(A[e]);
  const double s = block_sum(part, sh);
  if (threadIdx.x == 0) atomicAdd(acc, s);
}

template <typename C>
__global__ void __launch_bounds__(256) k_norm_apply(C* A, long long n, const double* acc, double* logscale) {
  const double nrm = sqrt(*acc);
  if (!(nrm > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *logscale = -INFINITY;
    return;
  }
  const double inv = 1.0 / nrm;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    A[e] = cscale(A[e], inv);
  if (blockIdx.x == 0 && threadIdx.x == 0) *logscale += log(nrm);
}

template <typename C>
__global__ void k_copy_tensor(const C* __restrict__ src, C* __restrict__ dst, int l, int p, int r, int tr) {
  long long tot = (long long)l * p * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    if (!tr) { dst[e] = src[e]; continue; }
    int a = (int)(e / ((long long)p * r));
    int q = (int)((e / r) % p);
    int b = (int)(e % r);
    dst[((long long)b * p + q) * l + a] = src[e];
  }
}

template <typename C>
__global__ void k_fill(C* A, long long n, double re, double im) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    A[e] = cx<C>(re, im);
}

template <typename C>
__global__ void k_conj_transpose(const C* __restrict__ src, int rows, int cols, C* __restrict__ dst) {
  long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / cols), j = (int)(e % cols);
    dst[(long long)j * rows + i] = cconj(src[e]);
  }
}

template <typename C>
__global__ void k_permute3(const C* __restrict__ src, int d0, int d1, int d2, int3 perm, C* __restrict__ dst) {
  const int dims[3] = {d0, d1, d2};
  const int pp[3] = {perm.x, perm.y, perm.z};
  const int od[3] = {dims[pp[0]], dims[pp[1]], dims[pp[2]]};
  long long tot = (long long)d0 * d1 * d2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int o[3];
    o[2] = (int)(e % od[2]);
    o[1] = (int)((e / od[2]) % od[1]);
    o[0] = (int)(e / ((long long)od[2] * od[1]));
    int sidx[3];
    for (int q = 0; q < 3; ++q) sidx[pp[q]] = o[q];
    dst[e] = src[((long long)sidx[0] * d1 + sidx[1]) * d2 + sidx[2]];
  }
}

// ---------------------------------------------------------------------- K4
// <M|M> by the transfer chain, <I|M> by the identity chain (both in
// complex128); the first tensor is scaled by |tr| / (tr sqrt(<M|M>)).
// One cluster of kK4Cluster CTAs: every phase of a transfer step splits its
// outputs over the cluster's threads and ends at a cluster barrier (the
// intermediates live in the global work buffer), so the complex128 work of
// one message runs on kK4Cluster SMs' FP64 units.
constexpr int kK4Cluster = 16;   // (a non-portable cluster size, opted in per kernel)
constexpr int kK4Split = 4;   // lanes per output of the r x r phase (divides 32)

template <typename C>
__global__ void __launch_bounds__(256) k_msg_normalise(ChainDesc d, double2* work) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
  const int tid = crank * blockDim.x + threadIdx.x, nth = csize * blockDim.x;
  double2* E = work;                   // l x l
  double2* E2 = work + 64 * 64;        // r x r
  double2* F = work + 2 * 64 * 64;     // l x p x r scratch
  double2* v = work + 2 * 64 * 64 + 64 * 64 * 64;   // identity chain (2 x 64), then the factor at v[128]
  if (tid == 0) { E[0] = make_double2(1.0, 0.0); v[0] = make_double2(1.0, 0.0); }
  cl.sync();
  for (int q = 0; q < d.k; ++q) {
    const int l = d.l[q], p = d.p[q], r = d.r[q];
    const C* A = (const C*)d.T[q];
    for (long long e = tid; e < (long long)l * p * r; e += nth) {
      int l2 = (int)(e / ((long long)p * r)), pp = (int)((e / r) % p), r1 = (int)(e % r);
      double2 s = make_double2(0.0, 0.0);
      for (int l1 = 0; l1 < l; ++l1) s = cadd(s, cmulc(c128(A[((long long)l1 * p + pp) * r + r1]), E[l1 * l + l2]));
      F[e] = s;
    }
    const int D = d.D[q];
    for (int e = tid; e < r; e += nth) {
      double2 s = make_double2(0.0, 0.0);
      for (int a = 0; a < l; ++a)
        for (int kk = 0; kk < D; ++kk) s = cadd(s, cmul(v[a], c128(A[((long long)a * p + kk * D + kk) * r + e])));
      v[64 + e] = s;
    }
    cl.sync();
    // r x r outputs of l p terms each: kK4Split consecutive lanes share one
    // output (strided terms, shuffle sum), so every thread has work
    for (int eb = (tid >> 5) * (32 / kK4Split); eb < r * r; eb += (nth >> 5) * (32 / kK4Split)) {
      const int e = eb + (threadIdx.x & 31) / kK4Split, sub = threadIdx.x % kK4Split;
      double2 s = make_double2(0.0, 0.0);
      if (e < r * r) {
        const int r1 = e / r, r2 = e % r;
        for (int t = sub; t < l * p; t += kK4Split)
          s = cadd(s, cmul(F[(long long)t * r + r1], c128(A[(long long)t * r + r2])));
      }
      for (int o = 1; o < kK4Split; o <<= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (e < r * r && sub == 0) E2[e] = s;
    }
    cl.sync();
    for (int e = tid; e < r * r; e += nth) E[e] = E2[e];
    for (int e = tid; e < r; e += nth) v[e] = v[64 + e];
    cl.sync();
  }
  if (tid == 0) {
    double nrm2 = E[0].x;
    double2 tr = v[0];
    double at = sqrt(tr.x * tr.x + tr.y * tr.y);
    double2 f = make_double2(nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 1.0, 0.0);
    if (at > 0.0) f = cmul(f, make_double2(tr.x / at, -tr.y / at));   // |tr| / tr
    v[128] = f;
  }
  cl.sync();
  const double2 f = v[128];
  C* T0 = (C*)d.T[0];
  const long long n0 = (long long)d.l[0] * d.p[0] * d.r[0];
  for (long long e = tid; e < n0; e += nth) {
    double2 x = cmul(c128(T0[e]), f);
    T0[e] = cx<C>(x.x, x.y);
  }
}

// direct sum of (a, -b) at chain position pos of k
template <typename C>
__global__ void k_direct_sum(const C* a, int la, int ra, const C* b, int lb, int rb, int p, int pos, int k, C* out) {
  int L = (k == 1 || pos == 0) ? 1 : la + lb;
  int R = (k == 1 || pos == k - 1) ? 1 : ra + rb;
  long long tot = (long long)L * p * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int x = (int)(e / ((long long)p * R)), q = (int)((e / R) % p), y = (int)(e % R);
    C v = cx<C>(0, 0);
    if (k == 1) {
      v = csub(a[q], b[q]);
    } else if (pos == 0) {
      if (y < ra) v = a[(long long)q * ra + y];
      else v = cscale(b[(long long)q * rb + (y - ra)], -1.0);
    } else if (pos == k - 1) {
      if (x < la) v = a[(long long)x * p + q];
      else v = b[(long long)(x - la) * p + q];
    } else {
      if (x < la && y < ra) v = a[((long long)x * p + q) * ra + y];
      else if (x >= la && y >= ra) v = b[((long long)(x - la) * p + q) * rb + (y - ra)];
    }
    out[e] = v;
  }
}

// The iteration's convergence word (Alg. 1 with the convergence criterion
// of the BP update): the largest message change over the nu updates, and
// flags: 1 a change is not finite, 2 a Jacobi reached its sweep limit, 4 a
// tensor-core wait timed out, 8 converged (largest change <= *tol, no other
// flag).  One CTA, after every update of the iteration has finished.
__global__ void __launch_bounds__(256) k_iter_reduce(const double* __restrict__ dist, const int* __restrict__ status,
                                                     int nu, const double* __restrict__ tol, double* __restrict__ out) {
  __shared__ double s_max[8];
  __shared__ int s_flags[8];
  double m = 0.0;
  int flags = 0;
  for (int u = threadIdx.x; u < nu; u += blockDim.x) {
    const double x = dist[u];
    if (!isfinite(x)) flags |= 1;
    else m = fmax(m, x);
    if (status[2 * u]) flags |= 2;
    if (status[2 * u + 1]) flags |= 4;
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_max[threadIdx.x >> 5] = m;
    s_flags[threadIdx.x >> 5] = flags;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, s_max[w]);
      flags |= s_flags[w];
    }
    if (!flags && m <= *tol) flags |= 8;
    out[0] = (flags & 1) ? NAN : m;
    ((int*)(out + 1))[0] = flags;
  }
}

// a x + b y as one MPS tensor at chain position pos of k: the direct sum of
// the bond spaces, the coefficients entering the first tensor (a single
// tensor is summed entrywise).  The learning step and the Hermitisation of
// a message (Sec. 2.3.3) add two MPSs this way.
template <typename C>
__global__ void k_mps_sum(const C* __restrict__ x, int lx, int rx, const C* __restrict__ y, int ly, int ry, int p,
                          int pos, int k, double2 ca, double2 cb, C* __restrict__ out) {
  const int L = (k == 1 || pos == 0) ? lx : lx + ly;
  const int R = (k == 1 || pos == k - 1) ? rx : rx + ry;
  const long long tot = (long long)L * p * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((long long)p * R)), q = (int)((e / R) % p), c = (int)(e % R);
    double2 v = make_double2(0.0, 0.0);
    if (k == 1) {
      v = cadd(cmul(ca, c128(x[e])), cmul(cb, c128(y[e])));
    } else if (pos == 0) {
      v = c < rx ? cmul(ca, c128(x[((long long)a * p + q) * rx + c])) : cmul(cb, c128(y[((long long)a * p + q) * ry + c - rx]));
    } else if (pos == k - 1) {
      v = a < lx ? c128(x[((long long)a * p + q) * rx + c]) : c128(y[((long long)(a - lx) * p + q) * ry + c]);
    } else if (a < lx && c < rx) {
      v = c128(x[((long long)a * p + q) * rx + c]);
    } else if (a >= lx && c >= rx) {
      v = c128(y[((long long)(a - lx) * p + q) * ry + c - rx]);
    }
    out[e] = cx<C>(v.x, v.y);
  }
}

// The message tensor read as an operator and Hermitian-conjugated: fused leg
// ket * D + bra becomes bra * D + ket, every entry conjugated.
template <typename C>
__global__ void k_mps_dagger(const C* __restrict__ src, int l, int D, int r, C* __restrict__ dst) {
  const long long tot = (long long)l * D * D * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % r);
    const long long t = e / r;
    const int j = (int)(t % D), i = (int)((t / D) % D), a = (int)(t / ((long long)D * D));
    dst[e] = cconj(src[(((long long)a * D + j) * D + i) * r + c]);
  }
}

template <typename C>
__global__ void __launch_bounds__(1024) k_frob(const C* R, long long n, double* out) {
  __shared__ double sh[40];
  double part = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) part += cabs2d(R[e]);
  double s = block_sum(part, sh);
  if (threadIdx.x == 0) *out = sqrt(s);
}

// value = sum prod A_q B_q over shared legs: E'[x][y] = sum_{i,j,p} E[i][j] a[i][p][x] b[j][p][y],
// in two steps through F[j][p][x] = sum_i E[i][j] a[i][p][x].  One cluster of
// kK4Cluster CTAs (phases separated by cluster barriers); work as for K4.
template <typename C>
__global__ void __launch_bounds__(256) k_mps_dot(ChainDesc A, ChainDesc B, double2* work, double2* out) {
  cg::cluster_group cl = cg::this_cluster();
  const int tid = (int)cl.block_rank() * blockDim.x + threadIdx.x, nth = (int)cl.num_blocks() * blockDim.x;
  double2* E = work;
  double2* E2 = work + 64 * 64;
  double2* F = work + 2 * 64 * 64;
  if (tid == 0) E[0] = make_double2(1.0, 0.0);
  cl.sync();
  for (int q = 0; q < A.k; ++q) {
    const int p = A.p[q], ra = A.r[q], rb = B.r[q];
    const int la = A.l[q], lb = B.l[q];
    const C* a = (const C*)A.T[q];
    const C* b = (const C*)B.T[q];
    for (long long e = tid; e < (long long)lb * p * ra; e += nth) {
      int j = (int)(e / ((long long)p * ra)), pp = (int)((e / ra) % p), x = (int)(e % ra);
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < la; ++i) s = cadd(s, cmul(E[i * lb + j], c128(a[((long long)i * p + pp) * ra + x])));
      F[e] = s;
    }
    cl.sync();
    for (int eb = (tid >> 5) * (32 / kK4Split); eb < ra * rb; eb += (nth >> 5) * (32 / kK4Split)) {
      const int e = eb + (threadIdx.x & 31) / kK4Split, sub = threadIdx.x % kK4Split;
      double2 s = make_double2(0.0, 0.0);
      if (e < ra * rb) {
        const int x = e / rb, y = e % rb;
        for (int t = sub; t < lb * p; t += kK4Split)
          s = cadd(s, cmul(F[(long long)t * ra + x], c128(b[(long long)t * rb + y])));
      }
      for (int o = 1; o < kK4Split; o <<= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (e < ra * rb && sub == 0) E2[e] = s;
    }
    cl.sync();
    for (int e = tid; e < ra * rb; e += nth) E[e] = E2[e];
    cl.sync();
  }
  if (tid == 0) *out = E[0];
}
}  // namespace

#define BBP_INSTANTIATE(C)                                                                                          \
  cudaError_t launch_normalise(C* A, long long n, double* logscale, cudaStream_t s) {                              \
    if (n <= (1 << 15)) {                                                                                          \
      k_normalise<C><<<1, 1024, 0, s>>>(A, n, logscale);                                                           \
      return cudaGetLastError();                                                                                   \
    }                                                                                                              \
    /* logscale[1]: the accumulator of the many-CTA form */                                                        \
    cudaError_t e = cudaMemsetAsync(logscale + 1, 0, sizeof(double), s);                                          \
    if (e != cudaSuccess) return e;                                                                                \
    const int g = (int)std::min<long long>((n + 2047) / 2048, 304);                                               \
    k_norm_sum<C><<<g, 256, 0, s>>>(A, n, logscale + 1);                                                           \
    k_norm_apply<C><<<g, 256, 0, s>>>(A, n, logscale + 1, logscale);                                               \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_copy_tensor(const C* src, C* dst, int l, int p, int r, bool transpose, cudaStream_t s) {       \
    k_copy_tensor<C><<<grid_for((long long)l * p * r, 256), 256, 0, s>>>(src, dst, l, p, r, transpose ? 1 : 0);    \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_fill(C* A, long long n, double re, double im, cudaStream_t s) {                               \
    k_fill<C><<<grid_for(n, 256), 256, 0, s>>>(A, n, re, im);                                                      \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_conj_transpose(const C* src, int rows, int cols, C* dst, cudaStream_t s) {                     \
    k_conj_transpose<C><<<grid_for((long long)rows * cols, 256), 256, 0, s>>>(src, rows, cols, dst);               \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_permute3(const C* src, int d0, int d1, int d2, const int perm[3], C* dst, cudaStream_t s) {   \
    k_permute3<C><<<grid_for((long long)d0 * d1 * d2, 256), 256, 0, s>>>(src, d0, d1, d2,                          \
                                                                      make_int3(perm[0], perm[1], perm[2]), dst);   \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_direct_sum(const C* a, int la, int ra, const C* b, int lb, int rb, int p, int pos, int k,     \
                                C* out, cudaStream_t s) {                                                          \
    long long tot = (long long)(la + lb) * p * (ra + rb);                                                          \
    k_direct_sum<C><<<grid_for(tot, 256), 256, 0, s>>>(a, la, ra, b, lb, rb, p, pos, k, out);                      \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_mps_sum(const C* x, int lx, int rx, const C* y, int ly, int ry, int p, int pos, int k,        \
                             double2 a, double2 b, C* out, cudaStream_t s) {                                        \
    const int L = (k == 1 || pos == 0) ? lx : lx + ly, R = (k == 1 || pos == k - 1) ? rx : rx + ry;                 \
    k_mps_sum<C><<<grid_for((long long)L * p * R, 256), 256, 0, s>>>(x, lx, rx, y, ly, ry, p, pos, k, a, b, out);  \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_mps_dagger(const C* src, int l, int D, int r, C* dst, cudaStream_t s) {                        \
    k_mps_dagger<C><<<grid_for((long long)l * D * D * r, 256), 256, 0, s>>>(src, l, D, r, dst);                    \
    return cudaGetLastError();                                                                                     \
  }                                                                                                                \
  cudaError_t launch_frob(const C* R, long long n, double* dist, cudaStream_t s) {                                 \
    k_frob<C><<<1, 1024, 0, s>>>(R, n, dist);                                                                      \
    return cudaGetLastError();                                                                                     \
  }

BBP_INSTANTIATE(double2)
BBP_INSTANTIATE(float2)

cudaError_t launch_iter_reduce(const double* dist, const int* status, int nu, const double* tol, double* out,
                               cudaStream_t s) {
  k_iter_reduce<<<1, 256, 0, s>>>(dist, status, nu, tol, out);
  return cudaGetLastError();
}

cudaError_t launch_msg_normalise(const ChainDesc& m, bool c64, double2* work, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kK4Cluster, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kK4Cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (c64) return cudaLaunchKernelEx(&cfg, k_msg_normalise<float2>, m, work);
  return cudaLaunchKernelEx(&cfg, k_msg_normalise<double2>, m, work);
}

cudaError_t launch_mps_dot(const ChainDesc& a, const ChainDesc& b, bool c64, double2* work, double2* out,
                           cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kK4Cluster, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kK4Cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (c64) return cudaLaunchKernelEx(&cfg, k_mps_dot<float2>, a, b, work, out);
  return cudaLaunchKernelEx(&cfg, k_mps_dot<double2>, a, b, work, out);
}

// Large-shared-memory opt-ins of every staged kernel on the current device
// (done once up front so that no attribute call falls inside a stream capture).
cudaError_t init_kernel_attributes() {
  cudaError_t e;
  if ((e = smem_optin<k_tsqr_smem<double2>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_tsqr_smem<float2>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_tsqr_reg<4>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_tsqr_reg<8>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_tsqr_reg<16>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_jacobi_smem<double2>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_jacobi_smem<float2>>()) != cudaSuccess) return e;
  if ((e = smem_optin<k_jacobi_cut64>()) != cudaSuccess) return e;
  for (const void* f : {(const void*)k_msg_normalise<double2>, (const void*)k_msg_normalise<float2>,
                        (const void*)k_mps_dot<double2>, (const void*)k_mps_dot<float2>,
                        (const void*)k_jacobi_cut64})
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
  if ((e = init_panel_attributes()) != cudaSuccess) return e;
  return init_tc_attributes();
}

}  // namespace bbp
