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

// sum of slot[off] over the cluster's CTAs in rank order (the same grouping
// in every CTA); remote loads are issued eight at a time before their additions
template <typename C>
__device__ __forceinline__ C cluster_sum(cg::cluster_group& cl, C* slot, size_t off, int cs) {
  C s = mkc<C>(0, 0);
  for (int q0 = 0; q0 < cs; q0 += 8) {
    C v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (q0 + u < cs) ? cl.map_shared_rank(slot, q0 + u)[off] : mkc<C>(0, 0);
#pragma unroll
    for (int u = 0; u < 8; ++u) s = padd(s, v[u]);
  }
  return s;
}

__device__ __forceinline__ double cluster_sum_d(cg::cluster_group& cl, double* slot, size_t off, int cs) {
  double s = 0.0;
  for (int q0 = 0; q0 < cs; q0 += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (q0 + u < cs) ? cl.map_shared_rank(slot, q0 + u)[off] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  return s;
}

// dynamic shared memory of one CTA: the column-major slice (n columns of
// ld = rows | 1 entries), two exchange slots of 2n entries (partial dots,
// row j), the gathered factors and row, tau, sc and the new diagonal of
// every step, and two partial norms
template <typename C>
__host__ __device__ inline size_t panel_smem(int rows, int n) {
  return sizeof(C) * ((size_t)(rows | 1) * n + 4 * (size_t)n + 2 * (size_t)n + 3 * (size_t)n) + 4 * sizeof(double) +
         64;
}

// Householder step j, with the cluster sums of step j already exchanged:
//  gather   threads c >= j read the sums (thread j forms the reflector)
//  pass     every warp forms the updated column j + 1 in registers from
//           the step's reflector and factor (x' = x - v f_{j+1}), updates
//           its columns c > j + 1 and, from the same registers, takes the
//           partial dots x'^H a_c of step j + 1; the warp of column j + 1
//           takes its partial norm and stores it after the cluster barrier
// (one block barrier and one cluster barrier per step).
// Column j stays unscaled while it is read as the reflector of step j; its
// warp scales it in the next step.  Rows of a CTA: lane l caches local rows
// l + 32 i, i < MAXR.
template <typename C, int MAXR>
__global__ void __launch_bounds__(kPanelThreads) k_panel_qr(const C* __restrict__ Ag, int m, int n, int rows,
                                                            C* __restrict__ Qg, C* __restrict__ Rg, long long stride) {
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  const long long panel = blockIdx.x / cs;
  Ag += panel * stride;
  if (Qg) Qg += panel * stride;
  if (Rg) Rg += panel * (long long)n * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = rows | 1;
  C* A = (C*)smem_raw;                   // local row t of column c at A[c * ld + t]
  C* slot = A + (size_t)ld * n;          // [2][2n]: partial dots (n), row j (n)
  C* gdot = slot + 4 * (size_t)n;        // gathered sums, then the factors f_c
  C* grow = gdot + n;                    // row j
  C* s_tau = grow + n;
  C* s_sc = s_tau + n;
  C* s_diag = s_sc + n;
  double* pnorm = (double*)(s_diag + n); // [2] partial squared norms
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r0 = cr * rows;
  const int mr = max(0, min(rows, m - r0));
  const int k = min(m, n);
  const C zero = mkc<C>(0, 0);

  for (long long e = threadIdx.x; e < (long long)mr * n; e += blockDim.x) {
    const int t = (int)(e / n), c = (int)(e % n);
    A[(size_t)c * ld + t] = Ag[(long long)(r0 + t) * n + c];
  }
  __syncthreads();

  auto load_col = [&](int c, C (&v)[MAXR]) {
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int t = lane + 32 * i;
      v[i] = t < mr ? A[(size_t)c * ld + t] : zero;
    }
  };
  auto store_col = [&](int c, const C (&v)[MAXR]) {
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int t = lane + 32 * i;
      if (t < mr) A[(size_t)c * ld + t] = v[i];
    }
  };
  // sum over this CTA's rows with global row > g0 of conj(x) y
  auto dot_below = [&](const C (&x)[MAXR], const C (&y)[MAXR], int g0) {
    C acc = zero;
#pragma unroll
    for (int i = 0; i < MAXR; ++i)
      if (r0 + lane + 32 * i > g0) acc = padd(acc, pmulc(x[i], y[i]));
    acc.x = wsum(acc.x);
    acc.y = wsum(acc.y);
    return acc;
  };
  auto norm_below = [&](const C (&x)[MAXR], int g0) {
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < MAXR; ++i)
      if (r0 + lane + 32 * i > g0 && lane + 32 * i < mr) s2 += (double)x[i].x * x[i].x + (double)x[i].y * x[i].y;
    return wsum(s2);
  };
  // row g of column values y into the exchange row when this CTA owns it
  auto put_row = [&](const C (&y)[MAXR], int g, C* dst) {
    const int t = g - r0;
    if (t < 0 || t >= mr) return;
#pragma unroll
    for (int i = 0; i < MAXR; ++i)
      if (lane + 32 * i == t) *dst = y[i];
  };

  // ---- factorisation
  if (k > 0) {                           // sums of step 0
    C x0[MAXR];
    load_col(0, x0);
    if (warp == 0) {
      const double s2 = norm_below(x0, 0);
      if (lane == 0) pnorm[0] = s2;
      put_row(x0, 0, slot + n + 0);
    }
    for (int c = 1 + warp; c < n; c += nw) {
      C y[MAXR];
      load_col(c, y);
      const C d = dot_below(x0, y, 0);
      if (lane == 0) slot[c] = d;
      put_row(y, 0, slot + n + c);
    }
  }
  cl.sync();
  for (int j = 0; j < k; ++j) {
    const int par = j & 1;
    const size_t off = (size_t)par * 2 * n, noff = (size_t)(par ^ 1) * 2 * n;
    const int owner = j / rows;
    for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
      grow[c] = cl.map_shared_rank(slot, owner)[off + n + c];
      if (c > j) {
        gdot[c] = cluster_sum(cl, slot, off + c, cs);
        continue;
      }
      const double xn2 = cluster_sum_d(cl, pnorm, par, cs);
      const C alpha = grow[j];
      double taur = 0, taui = 0, scr = 0, sci = 0, beta = alpha.x;
      const double ar = alpha.x, ai = alpha.y;
      if (!(xn2 == 0.0 && ai == 0.0)) {
        // beta from the norm accumulated in double; the remaining
        // parameters in the element's real type, with alpha - beta scaled by
        // 1 / |beta| (|alpha - beta| >= |beta|), so that nothing underflows
        using R = typename Real<C>::T;
        beta = -copysign(sqrt(ar * ar + ai * ai + xn2), ar);
        const R b = (R)beta, a_r = (R)ar, a_i = (R)ai;
        const R ib = (R)1 / b, sb = fabs(ib);
        const R dx = (a_r - b) * sb, dy = a_i * sb, idd = sb / (dx * dx + dy * dy);
        taur = (double)((b - a_r) * ib);
        taui = (double)(-a_i * ib);
        scr = (double)(dx * idd);
        sci = (double)(-dy * idd);
        // (the element type must hold sc too: columns near the bottom of its
        // range leave the column as it is)
        const double smax = sizeof(R) == 4 ? 1e37 : 1e300;
        if (!(isfinite(taur) && isfinite(taui) && isfinite(scr) && isfinite(sci) && isfinite(beta)) ||
            fabs(scr) > smax || fabs(sci) > smax || b == (R)0) {
          taur = taui = scr = sci = 0.0;
          beta = ar;
        }
      }
      const bool active = !(taur == 0.0 && taui == 0.0);
      s_tau[j] = mkc<C>(taur, taui);
      s_sc[j] = mkc<C>(scr, sci);
      s_diag[j] = mkc<C>(beta, active ? 0.0 : ai);
    }
    __syncthreads();
    const C tj = s_tau[j], sc = s_sc[j], ctau = mkc<C>(tj.x, -tj.y);
    const bool active = !(tj.x == 0 && tj.y == 0);
    // scale the reflector of step j - 1 (no longer read)
    if (j > 0 && warp == (j - 1) % nw) {
      C x[MAXR];
      load_col(j - 1, x);
      const C scp = s_sc[j - 1];
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const int g = r0 + lane + 32 * i;
        if (g > j - 1) x[i] = pmul(x[i], scp);
        else if (g == j - 1) x[i] = s_diag[j - 1];
      }
      store_col(j - 1, x);
    }
    C v[MAXR];                           // v of step j: x sc below row j, 1 at row j
    load_col(j, v);
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int g = r0 + lane + 32 * i;
      v[i] = g > j ? pmul(v[i], sc) : (g == j ? mkc<C>(1, 0) : zero);
    }
    auto fac = [&](int c) { return active ? pmul(ctau, padd(grow[c], pmulc(sc, gdot[c]))) : zero; };
    // one pass: every warp forms the updated column j + 1 in its registers
    // (x' = x - v f_{j+1}), updates its own columns c > j + 1 and takes the
    // partial dots x'^H a_c of step j + 1 from the same registers; the warp
    // of column j + 1 takes its partial norm, and stores it only after the
    // cluster barrier, when no warp reads the old column any more
    C xn[MAXR];
    const bool own_next = j + 1 < n && warp == (j + 1) % nw;
    if (j + 1 < n) {
      load_col(j + 1, xn);
      const C f1 = fac(j + 1);
#pragma unroll
      for (int i = 0; i < MAXR; ++i) xn[i] = psub(xn[i], pmul(v[i], f1));
      if (own_next) {
        if (j + 1 < k) {
          const double s2 = norm_below(xn, j + 1);
          if (lane == 0) pnorm[par ^ 1] = s2;
          put_row(xn, j + 1, slot + noff + n + j + 1);
        }
      }
      const int c0 = j + 2 + ((warp - (j + 2)) % nw + nw) % nw;
      for (int c = c0; c < n; c += nw) {
        C y[MAXR];
        load_col(c, y);
        const C f = fac(c);
#pragma unroll
        for (int i = 0; i < MAXR; ++i) y[i] = psub(y[i], pmul(v[i], f));
        store_col(c, y);
        if (j + 1 < k) {
          const C d = dot_below(xn, y, j + 1);
          if (lane == 0) slot[noff + c] = d;
          put_row(y, j + 1, slot + noff + n + c);
        }
      }
    }
    cl.sync();
    if (own_next) store_col(j + 1, xn);  // ordered before its reads by the next step's block barrier
  }
  if (k > 0 && warp == (k - 1) % nw) {   // scale the last reflector
    C x[MAXR];
    load_col(k - 1, x);
    const C scp = s_sc[k - 1];
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int g = r0 + lane + 32 * i;
      if (g > k - 1) x[i] = pmul(x[i], scp);
      else if (g == k - 1) x[i] = s_diag[k - 1];
    }
    store_col(k - 1, x);
  }
  __syncthreads();

  // R (k x n, upper triangular) from the rows this CTA holds
  if (Rg)
    for (long long e = threadIdx.x; e < (long long)mr * n; e += blockDim.x) {
      const int t = (int)(e / n), c = (int)(e % n), g = r0 + t;
      if (g < k) Rg[(long long)g * n + c] = (c >= g) ? A[(size_t)c * ld + t] : zero;
    }
  if (!Qg) return;     // no exchange slot is read after the last cl.sync above

  // ---- Q = H_0 ... H_{k-1} [I; 0], in place backwards: step i updates the
  // columns c > i by tau_i v_i (v_i^H q_c) and sets column i to
  // e_i - tau_i v_i; the pass of step i also takes the partial dots of step
  // i - 1 (v_{i-1} = column i - 1, untouched until its own step)
  auto refl = [&](int i, C (&x)[MAXR]) {  // v_i from column i (scaled, 1 on row i)
    load_col(i, x);
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int g = r0 + lane + 32 * q;
      x[q] = g > i ? x[q] : (g == i ? mkc<C>(1, 0) : zero);
    }
  };
  auto dot_from = [&](const C (&x)[MAXR], const C (&y)[MAXR]) {   // rows where x is nonzero
    C acc = zero;
#pragma unroll
    for (int q = 0; q < MAXR; ++q) acc = padd(acc, pmulc(x[q], y[q]));
    acc.x = wsum(acc.x);
    acc.y = wsum(acc.y);
    return acc;
  };
  auto set_col = [&](int i, const C (&x)[MAXR], C (&y)[MAXR]) {   // e_i - tau_i v_i
    const C ti = s_tau[i], mt = mkc<C>(-(double)ti.x, -(double)ti.y);
#pragma unroll
    for (int q = 0; q < MAXR; ++q) {
      const int g = r0 + lane + 32 * q;
      y[q] = g == i ? mkc<C>(1.0 - (double)ti.x, -(double)ti.y) : (g > i ? pmul(mt, x[q]) : zero);
    }
  };
  if (k > 0) {                           // column k - 1 and the sums of step k - 2
    C x[MAXR], xp[MAXR], y[MAXR];
    refl(k - 1, x);
    if (k >= 2) refl(k - 2, xp);
    __syncthreads();
    if (warp == (k - 1) % nw) {
      set_col(k - 1, x, y);
      store_col(k - 1, y);
      if (k >= 2) {
        const C d = dot_from(xp, y);
        if (lane == 0) slot[k - 1] = d;
      }
    }
  }
  cl.sync();
  for (int i = k - 2; i >= 0; --i) {
    const int par = (k - 2 - i) & 1;
    const size_t off = (size_t)par * 2 * n, noff = (size_t)(par ^ 1) * 2 * n;
    for (int c = i + 1 + threadIdx.x; c < k; c += blockDim.x)
      gdot[c] = pmul(s_tau[i], cluster_sum(cl, slot, off + c, cs));   // tau_i v_i^H q_c
    C x[MAXR], xp[MAXR];
    refl(i, x);
    if (i >= 1) refl(i - 1, xp);
    __syncthreads();                     // gdot complete; every warp holds v_i before column i changes
    for (int c = i + (((warp - i) % nw) + nw) % nw; c < k; c += nw) {
      C y[MAXR];
      if (c == i) {
        set_col(i, x, y);
      } else {
        load_col(c, y);
        const C f = gdot[c];
#pragma unroll
        for (int q = 0; q < MAXR; ++q) y[q] = psub(y[q], pmul(x[q], f));
      }
      store_col(c, y);
      if (i >= 1) {
        const C d = dot_from(xp, y);
        if (lane == 0) slot[noff + c] = d;
      }
    }
    cl.sync();
  }
  __syncthreads();
  for (long long e = threadIdx.x; e < (long long)mr * k; e += blockDim.x) {
    const int t = (int)(e / k), c = (int)(e % k);
    Qg[(long long)(r0 + t) * k + c] = A[(size_t)c * ld + t];
  }
}

constexpr int kPanelSmemMax = 211 * 1024;

template <typename C, int MAXR>
cudaError_t panel_optin_one() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_panel_qr<C, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_panel_qr<C, MAXR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <typename C>
cudaError_t panel_optin() {
  cudaError_t e;
  if ((e = panel_optin_one<C, 2>()) != cudaSuccess) return e;
  if ((e = panel_optin_one<C, 4>()) != cudaSuccess) return e;
  if constexpr (sizeof(C) == sizeof(float2)) return panel_optin_one<C, 8>();
  return cudaSuccess;
}

}  // namespace

cudaError_t init_panel_attributes() {
  cudaError_t e = panel_optin<float2>();
  if (e != cudaSuccess) return e;
  return panel_optin<double2>();
}

// Rows of one CTA are cached 32 x MAXR in registers: at most 256 (complex64)
// or 128 (complex128, twice the registers per entry) per CTA.
static int panel_max_rows(size_t elem) { return elem == sizeof(double2) ? 128 : 256; }

int panel_cluster(int m, int n, size_t elem) {
  if (m < n || n < 1) return 0;
  for (int cs = 1; cs <= kPanelMaxCluster; ++cs) {
    const int rows = (m + cs - 1) / cs;
    const size_t b = elem == sizeof(double2) ? panel_smem<double2>(rows, n) : panel_smem<float2>(rows, n);
    if (rows <= panel_max_rows(elem) && b <= (size_t)kPanelSmemMax) return cs;
  }
  return 0;
}

// Cluster size of a launch: the smallest that fits, raised so that no CTA
// holds more than kPanelRowsTarget rows (the per-column work of a CTA is its
// row slice times the trailing width; the exchange costs grow with the
// cluster).
int panel_cluster_auto(int m, int n, size_t elem) {
  const int cmin = panel_cluster(m, n, elem);
  if (cmin == 0) return 0;
  const int want = (m + kPanelRowsTarget - 1) / kPanelRowsTarget;
  return std::max(cmin, std::min(want, kPanelMaxCluster));
}

template <typename C>
static cudaError_t panel_t(const C* A, int m, int n, C* Q, C* R, int batch, long long stride, cudaStream_t s,
                           int cluster) {
  if (batch < 1 || m < 1 || n < 1) return cudaSuccess;
  const int cmin = panel_cluster(m, n, sizeof(C));
  if (cmin == 0 || cluster > kPanelMaxCluster || (cluster > 0 && cluster < cmin)) return cudaErrorInvalidValue;
  const int cs = cluster > 0 ? cluster : panel_cluster_auto(m, n, sizeof(C));
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
  if (rows <= 64) return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 2>, A, m, n, rows, Q, R, stride);
  if (rows <= 128) return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 4>, A, m, n, rows, Q, R, stride);
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (rows <= 256) return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 8>, A, m, n, rows, Q, R, stride);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_panel_qr(const float2* A, int m, int n, float2* Q, float2* R, int batch, long long stride,
                            cudaStream_t s, int cluster) {
  return panel_t(A, m, n, Q, R, batch, stride, s, cluster);
}
cudaError_t launch_panel_qr(const double2* A, int m, int n, double2* Q, double2* R, int batch, long long stride,
                            cudaStream_t s, int cluster) {
  return panel_t(A, m, n, Q, R, batch, stride, s, cluster);
}

}  // namespace bbp
