// FP64 complex kernels of the BlockBP message update (sm_103a).
//
//  K1 fuse           double-layer (ket-bra) tensor, Sec. 1.2 / Sec. 2.1
//  zgemm             complex GEMM used for merges, contractions and gauge moves
//  qr                Householder QR (canonical-form moves, Sec. 2.3.3)
//  K3 svd_trunc      truncated SVD by one-sided (row) Jacobi, keep chi (Sec. 1.1.1, 1.1.3)
//  K4 msg_*          message normalisation, phase and distance (Eq. of the BP
//                    convergence criterion; readings in the oracle / DESIGN)
//
// Large Jacobi problems run on a thread-block cluster (one matrix per
// cluster, cluster barriers between rounds); every loop is bounded.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace bbp {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double warp_sum(double v) {
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

// ------------------------------------------------------------------ K1 fuse

__global__ void k_fuse(const double2* __restrict__ t, int d, int Dfull, int4 n4, const double2* __restrict__ op,
                       int4 perm4, double2* __restrict__ T, long long total) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int nn[4] = {n4.x, n4.y, n4.z, n4.w};
  const int pp[4] = {perm4.x, perm4.y, perm4.z, perm4.w};
  int ket[4], bra[4];
  long long rem = idx;
  for (int q = 3; q >= 0; --q) {
    int leg = pp[q];
    int f2 = nn[leg] * nn[leg];
    int f = (int)(rem % f2);
    rem /= f2;
    ket[leg] = f / nn[leg];
    bra[leg] = f % nn[leg];
  }
  const long long D = Dfull;
  const long long sD4 = D * D * D * D;
  const long long ok = ((ket[0] * D + ket[1]) * D + ket[2]) * D + ket[3];
  const long long ob = ((bra[0] * D + bra[1]) * D + bra[2]) * D + bra[3];
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < d; ++s) {
    double2 tb = cconj(t[s * sD4 + ob]);
    if (op) {
      for (int sp = 0; sp < d; ++sp) acc = cadd(acc, cmul(op[s * d + sp], cmul(t[sp * sD4 + ok], tb)));
    } else {
      acc = cadd(acc, cmul(t[s * sD4 + ok], tb));
    }
  }
  T[idx] = acc;
}

// ------------------------------------------------------------------- zgemm

constexpr int GT = 32;   // output tile
constexpr int GK = 16;   // k tile

__device__ __forceinline__ double2 load_op(const double2* P, int ld, char op, int r, int c, int R, int C) {
  // element (r, c) of op(P), where op(P) is R x C
  if (r >= R || c >= C) return make_double2(0.0, 0.0);
  if (op == 'N') return P[(long long)r * ld + c];
  double2 v = P[(long long)c * ld + r];
  return op == 'C' ? cconj(v) : v;
}

__global__ void __launch_bounds__(256) k_zgemm(char opA, char opB, int M, int N, int K, double2 alpha,
                                               const double2* __restrict__ A, int lda, long long sA,
                                               const double2* __restrict__ B, int ldb, long long sB, double2 beta,
                                               double2* __restrict__ C, int ldc, long long sC) {
  __shared__ double2 As[GT][GK + 1];
  __shared__ double2 Bs[GK][GT + 1];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int i = e / GK, kk = e % GK;
      As[i][kk] = load_op(A, lda, opA, row0 + i, k0 + kk, M, K);
      int kb = e / GT, j = e % GT;
      Bs[kb][j] = load_op(B, ldb, opB, k0 + kb, col0 + j, K, N);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      double2 a0 = As[ty][kk], a1 = As[ty + 16][kk];
      double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
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
        double2 v = cmul(alpha, acc[i][j]);
        if (beta.x != 0.0 || beta.y != 0.0) v = cadd(v, cmul(beta, C[(long long)r * ldc + c]));
        C[(long long)r * ldc + c] = v;
      }
    }
}

// ---------------------------------------------------------------------- QR
// Householder with real diagonal of R (H = I - tau v v^H, v_j = 1).  One CTA;
// A (m x n, row-major, ld = n) is overwritten by R and the reflectors.

__device__ void cta_householder(double2* A, int m, int n, double2* tau, double* sh) {
  const int k = m < n ? m : n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double2 s_tau, s_scale;
  for (int j = 0; j < k; ++j) {
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) part += cabs2(A[(long long)i * n + j]);
    double xn2 = block_sum(part, sh);
    if (threadIdx.x == 0) {
      double2 alpha = A[(long long)j * n + j];
      if (xn2 == 0.0 && alpha.y == 0.0) {
        s_tau = make_double2(0.0, 0.0);
        s_scale = make_double2(0.0, 0.0);
      } else {
        double beta = -copysign(sqrt(cabs2(alpha) + xn2), alpha.x);
        s_tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        double2 den = make_double2(alpha.x - beta, alpha.y);     // 1 / (alpha - beta)
        double dd = cabs2(den);
        s_scale = make_double2(den.x / dd, -den.y / dd);
        A[(long long)j * n + j] = make_double2(beta, 0.0);
      }
      tau[j] = s_tau;
    }
    __syncthreads();
    const double2 tj = s_tau, sc = s_scale;
    if (tj.x == 0.0 && tj.y == 0.0) { __syncthreads(); continue; }
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[(long long)i * n + j] = cmul(A[(long long)i * n + j], sc);
    __syncthreads();
    // A[j:, c] -= conj(tau) v (v^H A[j:, c]) for c > j
    const double2 ctau = cconj(tj);
    for (int c = j + 1 + w; c < n; c += nw) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = j + lane; i < m; i += 32) {
        double2 v = (i == j) ? make_double2(1.0, 0.0) : A[(long long)i * n + j];
        s = cadd(s, cmulc(v, A[(long long)i * n + c]));
      }
      s.x = warp_sum(s.x);
      s.y = warp_sum(s.y);
      double2 f = cmul(ctau, s);
      for (int i = j + lane; i < m; i += 32) {
        double2 v = (i == j) ? make_double2(1.0, 0.0) : A[(long long)i * n + j];
        A[(long long)i * n + c] = csub(A[(long long)i * n + c], cmul(v, f));
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_qr(double2* A, int m, int n, double2* Q, double2* R, double2* tau) {
  __shared__ double sh[40];
  cta_householder(A, m, n, tau, sh);
  const int k = m < n ? m : n;
  for (long long e = threadIdx.x; e < (long long)k * n; e += blockDim.x) {
    int i = (int)(e / n), c = (int)(e % n);
    R[e] = (c >= i) ? A[(long long)i * n + c] : make_double2(0.0, 0.0);
  }
  for (long long e = threadIdx.x; e < (long long)m * k; e += blockDim.x) {
    int i = (int)(e / k), c = (int)(e % k);
    Q[e] = make_double2(i == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = k - 1; j >= 0; --j) {
    const double2 tj = tau[j];
    if (tj.x == 0.0 && tj.y == 0.0) continue;
    for (int c = j + w; c < k; c += nw) {
      double2 s = make_double2(0.0, 0.0);
      for (int i = j + lane; i < m; i += 32) {
        double2 v = (i == j) ? make_double2(1.0, 0.0) : A[(long long)i * n + j];
        s = cadd(s, cmulc(v, Q[(long long)i * k + c]));
      }
      s.x = warp_sum(s.x);
      s.y = warp_sum(s.y);
      double2 f = cmul(tj, s);
      for (int i = j + lane; i < m; i += 32) {
        double2 v = (i == j) ? make_double2(1.0, 0.0) : A[(long long)i * n + j];
        Q[(long long)i * k + c] = csub(Q[(long long)i * k + c], cmul(v, f));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- K3 Jacobi

struct SvdWork {
  double2* G;
  double2* WH;
  double* sigma;
  int* idx;
  int* counters;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__host__ __device__ inline SvdWork carve(void* work, int M, int N) {
  char* p = (char*)work;
  SvdWork w;
  w.G = (double2*)p; p += align256(sizeof(double2) * (size_t)M * N);
  w.WH = (double2*)p; p += align256(sizeof(double2) * (size_t)M * M);
  w.sigma = (double*)p; p += align256(sizeof(double) * (size_t)M);
  w.idx = (int*)p; p += align256(sizeof(int) * (size_t)M);
  w.counters = (int*)p;
  return w;
}

__global__ void k_svd_init(const double2* __restrict__ Z, int m, int n, SvdWork w) {
  const int M = m <= n ? m : n, N = m <= n ? n : m;
  long long tot = (long long)M * N, totw = (long long)M * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot + totw;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < tot) {
      int a = (int)(e / N), c = (int)(e % N);
      // rows of Z (m <= n) or rows of Z^H (m > n)
      w.G[e] = (m <= n) ? Z[(long long)a * n + c] : cconj(Z[(long long)c * n + a]);
    } else {
      long long f = e - tot;
      int a = (int)(f / M), c = (int)(f % M);
      w.WH[f] = make_double2(a == c ? 1.0 : 0.0, 0.0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) w.counters[threadIdx.x] = 0;
}

// Rotate rows a, b of G (length N) and of WH (length M) so that they become
// orthogonal.  Warp-cooperative; returns 1 when a rotation was applied.
__device__ int rotate_pair(double2* ra, double2* rb, int N, double2* wa, double2* wb, int M, int lane, double tol) {
  double al = 0.0, be = 0.0, gx = 0.0, gy = 0.0;
  for (int c = lane; c < N; c += 32) {
    double2 x = __ldcg(ra + c), y = __ldcg(rb + c);
    al += cabs2(x);
    be += cabs2(y);
    gx += x.x * y.x + x.y * y.y;      // x * conj(y)
    gy += x.y * y.x - x.x * y.y;
  }
  al = warp_sum(al);
  be = warp_sum(be);
  gx = warp_sum(gx);
  gy = warp_sum(gy);
  double g = sqrt(gx * gx + gy * gy);
  if (g == 0.0 || g <= tol * sqrt(al) * sqrt(be)) return 0;
  // rows whose norms differ by more than 1e30 do not affect each other at
  // working precision; rotating them only churns rounding noise (and never
  // meets the relative test once the small norm is subnormal)
  if (fmin(al, be) <= 1e-60 * fmax(al, be)) return 0;
  double2 e = make_double2(gx / g, gy / g);
  double zeta = (be - al) / (2.0 * g);
  double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
  for (int c = lane; c < N; c += 32) {
    double2 x = __ldcg(ra + c), y = __ldcg(rb + c);
    double2 ey = cmul(e, y);
    __stcg(ra + c, csub(cscale(x, cs), cscale(ey, sn)));
    __stcg(rb + c, cadd(cscale(x, sn), cscale(ey, cs)));
  }
  for (int c = lane; c < M; c += 32) {
    double2 x = __ldcg(wa + c), y = __ldcg(wb + c);
    double2 ey = cmul(e, y);
    __stcg(wa + c, csub(cscale(x, cs), cscale(ey, sn)));
    __stcg(wb + c, cadd(cscale(x, sn), cscale(ey, cs)));
  }
  return 1;
}

__global__ void __launch_bounds__(256) k_jacobi(SvdWork w, int M, int N, double tol, int max_sweeps, int* status) {
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
        rot += rotate_pair(w.G + (long long)a * N, w.G + (long long)b * N, N, w.WH + (long long)a * M,
                           w.WH + (long long)b * M, M, lane, tol);
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
    if (total == 0) return;
  }
  if (crank == 0 && threadIdx.x == 0) *status = 1;   // sweep limit reached
}

__global__ void k_row_norms(SvdWork w, int M, int N) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= M) return;
  double s = 0.0;
  for (int c = lane; c < N; c += 32) s += cabs2(w.G[(long long)row * N + c]);
  s = warp_sum(s);
  if (lane == 0) w.sigma[row] = sqrt(s);
}

__global__ void k_select(SvdWork w, int M, int k) {
  for (int a = threadIdx.x; a < M; a += blockDim.x) {
    double sa = w.sigma[a];
    int rank = 0;
    for (int b = 0; b < M; ++b) {
      double sb = w.sigma[b];
      rank += (sb > sa) || (sb == sa && b < a);
    }
    if (rank < k) w.idx[rank] = a;
  }
}

__global__ void k_svd_out(SvdWork w, int m, int n, int k, double2* __restrict__ U, double2* __restrict__ Rem) {
  const int M = m <= n ? m : n, N = m <= n ? n : m;
  long long totU = (long long)m * k, totR = (long long)k * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totU + totR;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < totU) {
      int i = (int)(e / k), r = (int)(e % k);
      int a = w.idx[r];
      if (m <= n) {
        U[e] = cconj(w.WH[(long long)a * M + i]);
      } else {
        double s = w.sigma[a];
        double smax = w.sigma[w.idx[0]];
        U[e] = s > 1e-30 * smax ? cscale(cconj(w.G[(long long)a * N + i]), 1.0 / s) : make_double2(0.0, 0.0);
      }
    } else {
      long long f = e - totU;
      int r = (int)(f / n), c = (int)(f % n);
      int a = w.idx[r];
      if (m <= n) Rem[f] = w.G[(long long)a * N + c];
      else Rem[f] = cscale(w.WH[(long long)a * M + c], w.sigma[a]);
    }
  }
}

// --------------------------------------------------------------- normalise

__global__ void __launch_bounds__(1024) k_normalise(double2* A, long long n, double* logscale) {
  __shared__ double sh[40];
  double part = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) part += cabs2(A[e]);
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

__global__ void k_copy_tensor(const double2* __restrict__ src, double2* __restrict__ dst, int l, int p, int r, int tr) {
  long long tot = (long long)l * p * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    if (!tr) { dst[e] = src[e]; continue; }
    int a = (int)(e / ((long long)p * r));
    int q = (int)((e / r) % p);
    int b = (int)(e % r);
    dst[((long long)b * p + q) * l + a] = src[e];
  }
}

__global__ void k_fill(double2* A, long long n, double re, double im) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    A[e] = make_double2(re, im);
}

// ---------------------------------------------------------------------- K4
// <M|M> by the transfer chain, <I|M> by the identity chain; the first tensor
// is scaled by |tr| / (tr sqrt(<M|M>)).  One CTA; work holds 2 chi^2 + chi*p*chi doubles2.
__global__ void __launch_bounds__(256) k_msg_normalise(double2* const* T, const int* shapes, int k, const int* Dleg,
                                                       double2* work) {
  __shared__ double2 s_fac;
  double2* E = work;                   // l x l
  double2* E2 = work + 64 * 64;        // r x r
  double2* F = work + 2 * 64 * 64;     // l x p x r scratch
  double2* v = work + 2 * 64 * 64 + 64 * 64 * 64;   // identity chain vectors (2 x 64)
  if (threadIdx.x == 0) { E[0] = make_double2(1.0, 0.0); v[0] = make_double2(1.0, 0.0); }
  __syncthreads();
  for (int q = 0; q < k; ++q) {
    const int l = shapes[3 * q], p = shapes[3 * q + 1], r = shapes[3 * q + 2];
    const double2* A = T[q];
    // F[l2][p][r1] = sum_l1 conj(A[l1][p][r1]) E[l1][l2]
    for (long long e = threadIdx.x; e < (long long)l * p * r; e += blockDim.x) {
      int l2 = (int)(e / ((long long)p * r)), pp = (int)((e / r) % p), r1 = (int)(e % r);
      double2 s = make_double2(0.0, 0.0);
      for (int l1 = 0; l1 < l; ++l1) s = cadd(s, cmulc(A[((long long)l1 * p + pp) * r + r1], E[l1 * l + l2]));
      F[e] = s;
    }
    // identity chain: v'[r] = sum_l v[l] sum_kk A[l][kk*D+kk][r]
    __syncthreads();
    const int D = Dleg[q];
    for (int e = threadIdx.x; e < r; e += blockDim.x) {
      double2 s = make_double2(0.0, 0.0);
      for (int a = 0; a < l; ++a)
        for (int kk = 0; kk < D; ++kk) s = cadd(s, cmul(v[a], A[((long long)a * p + kk * D + kk) * r + e]));
      v[64 + e] = s;
    }
    // E2[r1][r2] = sum_{l2,p} F[l2][p][r1] A[l2][p][r2]
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      int r1 = e / r, r2 = e % r;
      double2 s = make_double2(0.0, 0.0);
      for (int l2 = 0; l2 < l; ++l2)
        for (int pp = 0; pp < p; ++pp)
          s = cadd(s, cmul(F[((long long)l2 * p + pp) * r + r1], A[((long long)l2 * p + pp) * r + r2]));
      E2[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) E[e] = E2[e];
    for (int e = threadIdx.x; e < r; e += blockDim.x) v[e] = v[64 + e];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double nrm2 = E[0].x;
    double2 tr = v[0];
    double at = sqrt(cabs2(tr));
    double2 f = make_double2(nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 1.0, 0.0);
    if (at > 0.0) f = cmul(f, make_double2(tr.x / at, -tr.y / at));   // |tr| / tr
    s_fac = f;
  }
  __syncthreads();
  const double2 f = s_fac;
  const long long n0 = (long long)shapes[0] * shapes[1] * shapes[2];
  for (long long e = threadIdx.x; e < n0; e += blockDim.x) T[0][e] = cmul(T[0][e], f);
}

__global__ void k_direct_sum(const double2* a, int la, int ra, const double2* b, int lb, int rb, int p, int pos, int k,
                             double2* out) {
  // out = direct sum of (a, -b) at chain position pos of k
  int L = (k == 1 || pos == 0) ? 1 : la + lb;
  int R = (k == 1 || pos == k - 1) ? 1 : ra + rb;
  long long tot = (long long)L * p * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int x = (int)(e / ((long long)p * R)), q = (int)((e / R) % p), y = (int)(e % R);
    double2 v = make_double2(0.0, 0.0);
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

__global__ void __launch_bounds__(1024) k_frob(const double2* R, long long n, double* out) {
  __shared__ double sh[40];
  double part = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) part += cabs2(R[e]);
  double s = block_sum(part, sh);
  if (threadIdx.x == 0) *out = sqrt(s);
}

// value = sum prod A_q B_q (plain contraction of two MPS over shared physical legs)
__global__ void __launch_bounds__(256) k_mps_dot(double2* const* A, double2* const* B, const int* shA, const int* shB,
                                                 int k, double2* work, double2* out) {
  double2* E = work;                // la x lb
  double2* E2 = work + 64 * 64;
  if (threadIdx.x == 0) E[0] = make_double2(1.0, 0.0);
  __syncthreads();
  int la = 1, lb = 1;
  for (int q = 0; q < k; ++q) {
    const int p = shA[3 * q + 1], ra = shA[3 * q + 2], rb = shB[3 * q + 2];
    la = shA[3 * q];
    lb = shB[3 * q];
    const double2* a = A[q];
    const double2* b = B[q];
    for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) {
      int x = e / rb, y = e % rb;
      double2 s = make_double2(0.0, 0.0);
      for (int i = 0; i < la; ++i)
        for (int pp = 0; pp < p; ++pp) {
          double2 ai = a[((long long)i * p + pp) * ra + x];
          for (int j = 0; j < lb; ++j) s = cadd(s, cmul(cmul(E[i * lb + j], ai), b[((long long)j * p + pp) * rb + y]));
        }
      E2[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ra * rb; e += blockDim.x) E[e] = E2[e];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = E[0];
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

}  // namespace

// ------------------------------------------------------------------ launchers

cudaError_t launch_fuse(const double2* t, int d, int Dfull, const int n[4], const double2* op, const int perm[4],
                        double2* T, cudaStream_t s) {
  long long total = 1;
  for (int q = 0; q < 4; ++q) total *= (long long)n[q] * n[q];
  int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  k_fuse<<<(unsigned)blocks, threads, 0, s>>>(t, d, Dfull, make_int4(n[0], n[1], n[2], n[3]), op,
                                              make_int4(perm[0], perm[1], perm[2], perm[3]), T, total);
  return cudaGetLastError();
}

cudaError_t launch_zgemm(char opA, char opB, int M, int N, int K, double2 alpha, const double2* A, int lda,
                         long long strideA, const double2* B, int ldb, long long strideB, double2 beta, double2* C,
                         int ldc, long long strideC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, batch);
  k_zgemm<<<grid, 256, 0, s>>>(opA, opB, M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC);
  return cudaGetLastError();
}

cudaError_t launch_qr(double2* A, int m, int n, double2* Q, double2* R, double2* tau, cudaStream_t s) {
  k_qr<<<1, 256, 0, s>>>(A, m, n, Q, R, tau);
  return cudaGetLastError();
}

size_t svd_work_bytes(int m, int n) {
  size_t M = m < n ? m : n, N = m < n ? n : m;
  return align256(sizeof(double2) * M * N) + align256(sizeof(double2) * M * M) + align256(sizeof(double) * M) +
         align256(sizeof(int) * M) + 256;
}

cudaError_t launch_svd_trunc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work,
                             int* status, cudaStream_t s) {
  const int M = m < n ? m : n, N = m < n ? n : m;
  const int k = chi < M ? chi : M;
  SvdWork w = carve(work, M, N);
  k_svd_init<<<grid_for((long long)M * N + (long long)M * M, 256), 256, 0, s>>>(Z, m, n, w);
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
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_jacobi, w, M, N, 1e-14, 60, status);
  if (e != cudaSuccess) return e;
  k_row_norms<<<(M * 32 + 255) / 256, 256, 0, s>>>(w, M, N);
  k_select<<<1, 256, 0, s>>>(w, M, k);
  k_svd_out<<<grid_for((long long)m * k + (long long)k * n, 256), 256, 0, s>>>(w, m, n, k, U, Rem);
  return cudaGetLastError();
}

cudaError_t svd_stats(const void* work, int m, int n, int* sweeps, long long* rotations, cudaStream_t s) {
  const int M = m < n ? m : n, N = m < n ? n : m;
  SvdWork w = carve(const_cast<void*>(work), M, N);
  int c[4];
  cudaError_t e = cudaMemcpyAsync(c, w.counters, sizeof(c), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  *sweeps = c[2];
  *rotations = c[3];
  return e;
}

cudaError_t launch_normalise(double2* A, long long n, double* logscale, cudaStream_t s) {
  k_normalise<<<1, 1024, 0, s>>>(A, n, logscale);
  return cudaGetLastError();
}

cudaError_t launch_copy_tensor(const double2* src, double2* dst, int l, int p, int r, bool transpose, cudaStream_t s) {
  k_copy_tensor<<<grid_for((long long)l * p * r, 256), 256, 0, s>>>(src, dst, l, p, r, transpose ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_fill(double2* A, long long n, double re, double im, cudaStream_t s) {
  k_fill<<<grid_for(n, 256), 256, 0, s>>>(A, n, re, im);
  return cudaGetLastError();
}

cudaError_t launch_msg_normalise(double2* const* tensors, const int* shapes, int k, const int* Dleg, double* work,
                                 cudaStream_t s) {
  k_msg_normalise<<<1, 256, 0, s>>>(tensors, shapes, k, Dleg, (double2*)work);
  return cudaGetLastError();
}

cudaError_t launch_direct_sum(const double2* a, int la, int ra, const double2* b, int lb, int rb, int p, int pos,
                              int k, double2* out, cudaStream_t s) {
  long long tot = (long long)(la + lb) * p * (ra + rb);
  k_direct_sum<<<grid_for(tot, 256), 256, 0, s>>>(a, la, ra, b, lb, rb, p, pos, k, out);
  return cudaGetLastError();
}

cudaError_t launch_frob(const double2* R, long long n, double* dist, cudaStream_t s) {
  k_frob<<<1, 1024, 0, s>>>(R, n, dist);
  return cudaGetLastError();
}

cudaError_t launch_mps_dot(double2* const* A, double2* const* B, const int* shA, const int* shB, int k, double2* work,
                           double2* out, cudaStream_t s) {
  k_mps_dot<<<1, 256, 0, s>>>(A, B, shA, shB, k, work, out);
  return cudaGetLastError();
}

}  // namespace bbp

namespace bbp {
namespace {
__global__ void k_conj_transpose(const double2* __restrict__ src, int rows, int cols, double2* __restrict__ dst) {
  long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / cols), j = (int)(e % cols);
    double2 v = src[e];
    dst[(long long)j * rows + i] = make_double2(v.x, -v.y);
  }
}
__global__ void k_permute3(const double2* __restrict__ src, int d0, int d1, int d2, int3 perm, double2* __restrict__ dst) {
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
}  // namespace

cudaError_t launch_conj_transpose(const double2* src, int rows, int cols, double2* dst, cudaStream_t s) {
  long long n = (long long)rows * cols;
  int g = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  if (g < 1) g = 1;
  k_conj_transpose<<<g, 256, 0, s>>>(src, rows, cols, dst);
  return cudaGetLastError();
}

cudaError_t launch_permute3(const double2* src, int d0, int d1, int d2, const int perm[3], double2* dst, cudaStream_t s) {
  long long n = (long long)d0 * d1 * d2;
  int g = (int)std::min<long long>((n + 255) / 256, 152 * 16);
  if (g < 1) g = 1;
  k_permute3<<<g, 256, 0, s>>>(src, d0, d1, d2, make_int3(perm[0], perm[1], perm[2]), dst);
  return cudaGetLastError();
}
}  // namespace bbp
