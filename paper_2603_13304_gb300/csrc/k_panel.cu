// Householder QR of tall panels on a thread-block cluster (Sec. 2.3.3: the
// canonical moves and the orthonormalisations of the truncation).
//
// A panel A (m x n, m >= n, row-major) is cut into cs contiguous row slices,
// one per CTA of a cluster of cs <= 16 CTAs; each slice stays in that CTA's
// shared memory for the whole factorisation.  Householder step j needs three
// sums over all rows below the diagonal: the squared norm of column j, and
// x^H a_c for every trailing column c (x = column j below row j).  Because
// the reflector is v = [1; x / (alpha - beta)], v^H a_c = a_jc + conj(sc)
// x^H a_c follows from those raw sums and row j, so one cluster-wide
// exchange per column suffices: every CTA writes its partial sums (and the
// owner of row j writes row j) into a double-buffered slot of its shared
// memory, the cluster synchronises once, and every CTA reads all slots
// through distributed shared memory and forms the same reflector in the same
// order (bitwise identical in every CTA).  Q = H_0 ... H_{k-1} [I; 0] is
// then formed in place backwards with one exchange per reflector.
//
// Convention (the same as the one-CTA kernels): H = I - tau v v^H, v_j = 1,
// R has a real diagonal beta_j, the factorisation applies H_j^H.  Norms are
// accumulated in double in both precisions, so complex64 columns neither
// underflow nor overflow when squared.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace bbp {

namespace {

template <typename C> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

template <typename C> __device__ __forceinline__ C mkc(double re, double im);
template <> __device__ __forceinline__ double2 mkc(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 mkc(double re, double im) { return make_float2((float)re, (float)im); }

template <typename C> __device__ __forceinline__ C pmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C pmulc(C a, C b) {   // conj(a) * b
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C padd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C psub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }

template <typename R> __device__ __forceinline__ R wsum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kPanelThreads = 512;

// sum of slot[off] over the cluster's CTAs in rank order; the remote loads
// are issued together before the additions
template <typename C>
__device__ __forceinline__ C cluster_sum(cg::cluster_group& cl, C* slot, size_t off, int cs) {
  C v[kPanelMaxCluster];
#pragma unroll
  for (int q = 0; q < kPanelMaxCluster; ++q)
    if (q < cs) v[q] = cl.map_shared_rank(slot, q)[off];
  C s = mkc<C>(0, 0);
#pragma unroll
  for (int q = 0; q < kPanelMaxCluster; ++q)
    if (q < cs) s = padd(s, v[q]);
  return s;
}

// dynamic shared memory of one CTA: slice (rows x (n + 1)), two exchange
// slots of 2n entries (partial dots, row j), the gathered dots and row, tau,
// and two partial norms
template <typename C>
__host__ __device__ inline size_t panel_smem(int rows, int n) {
  return sizeof(C) * ((size_t)rows * (n + 1) + 4 * (size_t)n + 2 * (size_t)n + (size_t)n) + 4 * sizeof(double) + 64;
}

template <typename C>
__global__ void __launch_bounds__(kPanelThreads) k_panel_qr(const C* __restrict__ Ag, int m, int n, int rows,
                                                            C* __restrict__ Qg, C* __restrict__ Rg, long long stride) {
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  const long long panel = blockIdx.x / cs;
  Ag += panel * stride;
  if (Qg) Qg += panel * stride;
  if (Rg) Rg += panel * (long long)n * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = n + 1;
  C* A = (C*)smem_raw;                   // local row i (global r0 + i), column c at A[i * ld + c]
  C* slot = A + (size_t)rows * ld;       // [2][2n]: partial dots (n), row j (n)
  C* gdot = slot + 4 * (size_t)n;        // gathered sums
  C* grow = gdot + n;
  C* s_tau = grow + n;
  double* pnorm = (double*)(s_tau + n);  // [2] partial squared norms
  double* gnorm = pnorm + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r0 = cr * rows;
  const int mr = max(0, min(rows, m - r0));
  const int k = min(m, n);

  for (long long e = threadIdx.x; e < (long long)mr * n; e += blockDim.x) {
    const int i = (int)(e / n), c = (int)(e % n);
    A[(size_t)i * ld + c] = Ag[(long long)(r0 + i) * n + c];
  }
  __syncthreads();

  // partial sums of step j into slot `par`: warps over columns c >= j
  // (c == j: the squared norm), lanes over local rows with global row > j
  auto partials = [&](int j, int par) {
    C* sd = slot + (size_t)par * 2 * n;
    const int i0 = max(0, j + 1 - r0);
    for (int c = j + warp; c < n; c += nw) {
      if (c == j) {
        double s = 0.0;
        for (int i = i0 + lane; i < mr; i += 32) {
          const C x = A[(size_t)i * ld + j];
          s += (double)x.x * x.x + (double)x.y * x.y;
        }
        s = wsum(s);
        if (lane == 0) pnorm[par] = s;
      } else {
        C acc = mkc<C>(0, 0);
        for (int i = i0 + lane; i < mr; i += 32) acc = padd(acc, pmulc(A[(size_t)i * ld + j], A[(size_t)i * ld + c]));
        acc.x = wsum(acc.x);
        acc.y = wsum(acc.y);
        if (lane == 0) sd[c] = acc;
      }
    }
    if (j >= r0 && j < r0 + mr)          // owner of row j
      for (int c = j + threadIdx.x; c < n; c += blockDim.x) sd[n + c] = A[(size_t)(j - r0) * ld + c];
  };

  if (k > 0) partials(0, 0);
  cl.sync();
  for (int j = 0; j < k; ++j) {
    const int par = j & 1;
    const int owner = j / rows;
    // gather the cluster's sums (identical order in every CTA)
    for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
      if (c > j) gdot[c] = cluster_sum(cl, slot, (size_t)par * 2 * n + c, cs);
      grow[c] = cl.map_shared_rank(slot, owner)[(size_t)par * 2 * n + n + c];
    }
    if (threadIdx.x == blockDim.x - 1) {
      double s = 0.0;
      for (int q = 0; q < cs; ++q) s += cl.map_shared_rank(pnorm, q)[par];
      *gnorm = s;
    }
    __syncthreads();
    // reflector (every thread, same arithmetic)
    const double xn2 = *gnorm;
    const C alpha = grow[j];
    double taur = 0, taui = 0, scr = 0, sci = 0, beta = alpha.x;
    const double ar = alpha.x, ai = alpha.y;
    if (!(xn2 == 0.0 && ai == 0.0)) {
      beta = -copysign(sqrt(ar * ar + ai * ai + xn2), ar);
      taur = (beta - ar) / beta;
      taui = -ai / beta;
      const double dx = ar - beta, dy = ai, dd = dx * dx + dy * dy;
      scr = dx / dd;
      sci = -dy / dd;
      // (the element type must hold sc too: complex64 columns near the
      // bottom of the float range leave the column as it is)
      const double smax = sizeof(typename Real<C>::T) == 4 ? 1e37 : 1e300;
      if (!(isfinite(taur) && isfinite(taui) && isfinite(scr) && isfinite(sci) && isfinite(beta)) ||
          fabs(scr) > smax || fabs(sci) > smax) {
        taur = taui = scr = sci = 0.0;
        beta = ar;
      }
    }
    const C sc = mkc<C>(scr, sci);
    const C ctau = mkc<C>(taur, -taui);
    const bool active = !(taur == 0.0 && taui == 0.0);
    if (threadIdx.x == 0) s_tau[j] = mkc<C>(taur, taui);
    // update: a warp per local row, lanes over the trailing columns
    for (int i = warp; i < mr; i += nw) {
      const int gr = r0 + i;
      if (gr < j) continue;
      C* row = A + (size_t)i * ld;
      if (gr == j) {
        for (int c = j + 1 + lane; c < n; c += 32) {
          const C f = active ? pmul(ctau, padd(grow[c], pmulc(sc, gdot[c]))) : mkc<C>(0, 0);
          row[c] = psub(grow[c], f);
        }
        if (lane == 0) row[j] = mkc<C>(beta, active ? 0.0 : ai);
      } else if (active) {
        const C x = row[j];
        const C v = pmul(x, sc);
        for (int c = j + 1 + lane; c < n; c += 32) {
          const C f = pmul(ctau, padd(grow[c], pmulc(sc, gdot[c])));
          row[c] = psub(row[c], pmul(v, f));
        }
        __syncwarp();
        if (lane == 0) row[j] = v;
      }
    }
    __syncthreads();
    if (j + 1 < k) partials(j + 1, par ^ 1);
    cl.sync();
  }

  // R (k x n, upper triangular) from the rows this CTA holds
  if (Rg)
    for (long long e = threadIdx.x; e < (long long)mr * n; e += blockDim.x) {
      const int i = (int)(e / n), c = (int)(e % n), gr = r0 + i;
      if (gr < k) Rg[(long long)gr * n + c] = (c >= gr) ? A[(size_t)i * ld + c] : mkc<C>(0, 0);
    }
  if (!Qg) return;     // no exchange slot is read after the last cl.sync above
  __syncthreads();

  // Q backwards: step i needs v_i^H q_c over all rows for c in (i, k)
  auto qpartials = [&](int i, int par) {
    C* sd = slot + (size_t)par * 2 * n;
    const int i0 = max(0, i - r0);
    for (int c = i + 1 + warp; c < k; c += nw) {
      C acc = mkc<C>(0, 0);
      for (int t = i0 + lane; t < mr; t += 32) {
        const int gr = r0 + t;
        const C v = (gr == i) ? mkc<C>(1, 0) : A[(size_t)t * ld + i];
        acc = padd(acc, pmulc(v, A[(size_t)t * ld + c]));
      }
      acc.x = wsum(acc.x);
      acc.y = wsum(acc.y);
      if (lane == 0) sd[c] = acc;
    }
  };
  if (k > 0) qpartials(k - 1, 0);
  cl.sync();
  for (int i = k - 1; i >= 0; --i) {
    const int par = (k - 1 - i) & 1;
    for (int c = i + 1 + threadIdx.x; c < k; c += blockDim.x) {
      gdot[c] = cluster_sum(cl, slot, (size_t)par * 2 * n + c, cs);
    }
    __syncthreads();
    const C ti = s_tau[i];
    for (int t = warp; t < mr; t += nw) {
      const int gr = r0 + t;
      C* row = A + (size_t)t * ld;
      const C v = (gr == i) ? mkc<C>(1, 0) : (gr > i ? row[i] : mkc<C>(0, 0));
      if (gr >= i)
        for (int c = i + 1 + lane; c < k; c += 32) row[c] = psub(row[c], pmul(v, pmul(ti, gdot[c])));
      __syncwarp();
      if (lane == 0) {
        // column i := e_i - tau_i v_i
        if (gr == i) row[i] = mkc<C>(1.0 - (double)ti.x, -(double)ti.y);
        else if (gr > i) row[i] = pmul(mkc<C>(-(double)ti.x, -(double)ti.y), v);
        else row[i] = mkc<C>(0, 0);
      }
    }
    __syncthreads();
    if (i > 0) qpartials(i - 1, par ^ 1);
    cl.sync();
  }
  for (long long e = threadIdx.x; e < (long long)mr * k; e += blockDim.x) {
    const int t = (int)(e / k), c = (int)(e % k);
    Qg[(long long)(r0 + t) * k + c] = A[(size_t)t * ld + c];
  }
}

constexpr int kPanelSmemMax = 211 * 1024;

template <typename C>
cudaError_t panel_optin() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_panel_qr<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_panel_qr<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

}  // namespace

cudaError_t init_panel_attributes() {
  cudaError_t e = panel_optin<float2>();
  if (e != cudaSuccess) return e;
  return panel_optin<double2>();
}

int panel_cluster(int m, int n, size_t elem) {
  if (m < n || n < 1) return 0;
  for (int cs = 1; cs <= kPanelMaxCluster; ++cs) {
    const int rows = (m + cs - 1) / cs;
    const size_t b = elem == sizeof(double2) ? panel_smem<double2>(rows, n) : panel_smem<float2>(rows, n);
    if (b <= (size_t)kPanelSmemMax) return cs;
  }
  return 0;
}

template <typename C>
static cudaError_t panel_t(const C* A, int m, int n, C* Q, C* R, int batch, long long stride, cudaStream_t s) {
  if (batch < 1 || m < 1 || n < 1) return cudaSuccess;
  const int cs = panel_cluster(m, n, sizeof(C));
  if (cs == 0) return cudaErrorInvalidValue;
  cudaError_t e = panel_optin<C>();
  if (e != cudaSuccess) return e;
  const int rows = (m + cs - 1) / cs;
  KTimerScope timer(KC_ORTH, s, batch * qr_flops(m, n));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs * batch, 1, 1);
  cfg.blockDim = dim3(kPanelThreads, 1, 1);
  cfg.dynamicSmemBytes = panel_smem<C>(rows, n);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_panel_qr<C>, A, m, n, rows, Q, R, stride);
}

cudaError_t launch_panel_qr(const float2* A, int m, int n, float2* Q, float2* R, int batch, long long stride,
                            cudaStream_t s) {
  return panel_t(A, m, n, Q, R, batch, stride, s);
}
cudaError_t launch_panel_qr(const double2* A, int m, int n, double2* Q, double2* R, int batch, long long stride,
                            cudaStream_t s) {
  return panel_t(A, m, n, Q, R, batch, stride, s);
}

}  // namespace bbp
