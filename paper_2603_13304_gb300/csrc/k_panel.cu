// Householder QR of tall panels on a thread-block cluster (Sec. 2.3.3: the
// canonical moves and the orthonormalisations of the truncation).
//
// A panel A (m x n, m >= n, row-major) is cut into row slices of 32 MAXR
// rows, one per CTA of a cluster of cs <= 16 CTAs; each slice stays in that
// CTA's shared memory (column-major, zero-padded to 32 MAXR rows) for the
// whole factorisation, and lane l of a warp caches rows l + 32 i of the
// columns it works on.  Householder step j needs three sums over all rows
// below the diagonal: the squared norm of column j, and x^H a_c for every
// trailing column c (x = column j below row j).  Because the reflector is
// v = [1; x / (alpha - beta)], v^H a_c = a_jc + conj(sc) x^H a_c follows from
// those raw sums and row j, so one cluster-wide exchange per column
// suffices.  The exchange is pushed: every CTA stores its partial sums (and
// the owner of row j stores row j) straight into every CTA's receive buffer
// in distributed shared memory before the cluster barrier, so that after it
// every CTA reads only its own shared memory and forms the same reflector
// from the same values in the same order (bitwise identical in every CTA).
// Q = H_0 ... H_{k-1} [I; 0] is then formed in place backwards with one
// exchange per reflector.
//
// Convention (the same as the one-CTA kernels): H = I - tau v v^H, v_j = 1,
// R has a real diagonal beta_j, the factorisation applies H_j^H.  Column
// norms are exchanged as (power-of-two scale, scaled sum of squares) pairs in
// the element's real type, so complex64 columns neither overflow nor
// underflow when squared and the complex64 kernel does no FP64 arithmetic.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <initializer_list>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace bbp {

namespace {

template <typename C> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

template <typename C> __device__ __forceinline__ C mkc(typename Real<C>::T re, typename Real<C>::T im) {
  C r;
  r.x = re;
  r.y = im;
  return r;
}

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
template <typename R> __device__ __forceinline__ R wmax(R v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// y[q] for a warp-uniform q, by bit masks (a select chain here is turned
// into an indexed access, which puts the array in local memory)
template <int MAXR>
__device__ __forceinline__ float2 pick(const float2 (&y)[MAXR], int q) {
  unsigned a = 0, b = 0;
#pragma unroll
  for (int i = 0; i < MAXR; ++i) {
    const unsigned msk = q == i ? ~0u : 0u;
    a |= msk & __float_as_uint(y[i].x);
    b |= msk & __float_as_uint(y[i].y);
  }
  return make_float2(__uint_as_float(a), __uint_as_float(b));
}
template <int MAXR>
__device__ __forceinline__ double2 pick(const double2 (&y)[MAXR], int q) {
  unsigned long long a = 0, b = 0;
#pragma unroll
  for (int i = 0; i < MAXR; ++i) {
    const unsigned long long msk = q == i ? ~0ull : 0ull;
    a |= msk & (unsigned long long)__double_as_longlong(y[i].x);
    b |= msk & (unsigned long long)__double_as_longlong(y[i].y);
  }
  return make_double2(__longlong_as_double((long long)a), __longlong_as_double((long long)b));
}

constexpr int kPanelThreads = 512;
constexpr int kPanelSmemMax = 227 * 1024;
constexpr int kQBlock = 8;               // reflectors a block of the Q formation

// distributed shared memory through 32-bit shared-window addresses
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t dsmem_addr(uint32_t a, int rank) {
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_dsmem(uint32_t a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_dsmem(uint32_t a, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

// Shared memory of one CTA, in elements: the slice (n columns of ld >= 32
// MAXR entries), the receive buffers of the partial sums ([2][cs][n], by
// step parity and source CTA), row j ([2][n]), the gathered sums (n, when
// staged), the partial norms ([2][cs]), tau of every step (n, when Q is
// formed) and tau, sc and the new diagonal of the last two steps.
struct PanelLayout {
  int ld;
  size_t recv, rowb, gs, pp, tau, ring, bytes;
};
template <typename C>
__host__ __device__ inline PanelLayout panel_layout(int maxr, int n, int cs, bool want_q, bool odd_ld, bool gs) {
  PanelLayout L;
  L.ld = 32 * maxr + (odd_ld ? 1 : 0);
  size_t o = (size_t)L.ld * n;
  const size_t ex0 = o;
  L.recv = o; o += 2 * (size_t)cs * n;
  L.rowb = o; o += 2 * (size_t)n;
  L.gs = o; o += gs ? (size_t)n : 0;
  L.pp = o; o += 2 * (size_t)cs;
  // the same area holds the block buffers of the Q formation
  if (want_q) {
    const size_t qb = ex0 + 3 * (size_t)kQBlock * (n + kQBlock) + (size_t)kQBlock * kQBlock;
    o = o > qb ? o : qb;
  }
  L.tau = o; o += want_q ? (size_t)n : 0;
  L.ring = o; o += 6;
  L.bytes = sizeof(C) * o;
  return L;
}

// Householder step j, with the partial sums of step j already received:
//  gather   threads c > j sum the received partial dots of column c (in
//           source order); one thread forms the reflector from the partial
//           norms and row j
//  pass     every warp forms the updated column j + 1 in registers from the
//           step's reflector and factor (x' = x - v f_{j+1}), updates its
//           columns c > j + 1 and, from the same registers, takes the
//           partial dots x'^H a_c of step j + 1 and pushes them (and row
//           j + 1, from its owner CTA) to every CTA; the warp of column j + 1
//           pushes its partial norm and stores the column after the cluster
//           barrier, when no warp reads the old one any more
// (one block barrier and one cluster barrier per step).  Column c is always
// worked on by warp c mod nw, so a warp's own deferred stores and later loads
// of a column are ordered by program order.  Column j stays unscaled while it
// is read as the reflector of step j; its warp scales it in the next step.
template <typename C, int MAXR>
__global__ void __launch_bounds__(kPanelThreads, 1) k_panel_qr(const C* __restrict__ Ag, int m, int n,
                                                            C* __restrict__ Qg, C* __restrict__ Rg, long long stride,
                                                            int ld, int use_gs) {
  using R = typename Real<C>::T;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  const long long panel = blockIdx.x / cs;
  Ag += panel * stride;
  if (Qg) Qg += panel * stride;
  if (Rg) Rg += panel * (long long)n * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PanelLayout L = panel_layout<C>(MAXR, n, cs, Qg != nullptr, (ld & 1) != 0, use_gs != 0);
  C* A = (C*)smem_raw;                   // local row t of column c at A[c * ld + t]
  C* recv = A + L.recv;
  C* rowb = A + L.rowb;
  C* gs = A + L.gs;
  C* pp = A + L.pp;                      // (scale, scaled sum of squares)
  C* s_tau = A + L.tau;
  C* ring = A + L.ring;                  // [2][3]: tau, sc, diagonal
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int rows = 32 * MAXR;
  const int r0 = cr * rows;
  const int mr = max(0, min(rows, m - r0));
  const int k = min(m, n);
  const C zero = mkc<C>(0, 0), one = mkc<C>(1, 0);
  // lane q < cs pushes to CTA q
  const uint32_t recv_q = lane < cs ? dsmem_addr(smem_addr(recv), lane) : 0u;
  const uint32_t rowb_q = lane < cs ? dsmem_addr(smem_addr(rowb), lane) : 0u;
  const uint32_t pp_q = lane < cs ? dsmem_addr(smem_addr(pp), lane) : 0u;

  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int t = e / n, c = e % n;
    A[(size_t)c * ld + t] = t < mr ? Ag[(long long)(r0 + t) * n + c] : zero;
  }
  cl.sync();                             // every CTA of the cluster runs before the first push

  auto load_col = [&](int c, C (&v)[MAXR]) {
    const C* p = A + (size_t)c * ld + lane;
#pragma unroll
    for (int i = 0; i < MAXR; ++i) v[i] = p[32 * i];
  };
  auto store_col = [&](int c, const C (&v)[MAXR]) {
    C* p = A + (size_t)c * ld + lane;
#pragma unroll
    for (int i = 0; i < MAXR; ++i) p[32 * i] = v[i];
  };
  auto mask_below = [&](C (&x)[MAXR], int g0) {   // keep global rows > g0
#pragma unroll
    for (int i = 0; i < MAXR; ++i)
      if (r0 + lane + 32 * i <= g0) x[i] = zero;
  };
  auto dot = [&](const C (&x)[MAXR], const C (&y)[MAXR]) {   // sum over the slice of conj(x) y
    C acc = pmulc(x[0], y[0]);
#pragma unroll
    for (int i = 1; i < MAXR; ++i) acc = padd(acc, pmulc(x[i], y[i]));
    acc.x = wsum(acc.x);
    acc.y = wsum(acc.y);
    return acc;
  };
  // (scale, sum of squares / scale^2) of the slice; complex128: (1, sum)
  auto norm_part = [&](const C (&x)[MAXR]) {
    if constexpr (sizeof(R) == 8) {
      R s2 = 0;
#pragma unroll
      for (int i = 0; i < MAXR; ++i) s2 += x[i].x * x[i].x + x[i].y * x[i].y;
      return mkc<C>(1, wsum(s2));
    } else {
      R amax = 0;
#pragma unroll
      for (int i = 0; i < MAXR; ++i) amax = fmaxf(amax, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
      amax = wmax(amax);
      if (amax == 0) return zero;
      int ex;
      frexpf(amax, &ex);                 // amax < 2^ex; 2^-ex in two in-range factors
      const R s1 = ldexpf(1.f, -(ex / 2)), s2 = ldexpf(1.f, -(ex - ex / 2));
      R ss = 0;
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const R a = x[i].x * s1 * s2, b = x[i].y * s1 * s2;
        ss += a * a + b * b;
      }
      return mkc<C>(ldexpf(1.f, ex), wsum(ss));
    }
  };
  auto push_recv = [&](int par, int c, C d) {
    if (lane < cs) st_dsmem(recv_q + (uint32_t)(sizeof(C) * ((size_t)(par * cs + cr) * n + c)), d);
  };
  auto push_norm = [&](int par, C np) {
    if (lane < cs) st_dsmem(pp_q + (uint32_t)(sizeof(C) * (size_t)(par * cs + cr)), np);
  };
  // row g of column values y, from the CTA that holds it, into every CTA
  auto push_row = [&](const C (&y)[MAXR], int g, int par, int c) {
    const int t = g - r0;
    if (t < 0 || t >= mr) return;        // uniform over the CTA
    C val = pick(y, t >> 5);
    val.x = __shfl_sync(0xffffffffu, val.x, t & 31);
    val.y = __shfl_sync(0xffffffffu, val.y, t & 31);
    if (lane < cs) st_dsmem(rowb_q + (uint32_t)(sizeof(C) * ((size_t)par * n + c)), val);
  };
  auto sum_recv = [&](int par, int c) {   // the cluster sum of column c, in source order
    C s = zero;
    for (int q = 0; q < cs; ++q) s = padd(s, recv[(size_t)(par * cs + q) * n + c]);
    return s;
  };

  // ---- factorisation
  if (k > 0) {                           // sums of step 0
    C x[MAXR];
    load_col(0, x);
    if (warp == 0) push_row(x, 0, 0, 0);
    mask_below(x, 0);
    if (warp == 0) push_norm(0, norm_part(x));
    for (int c = warp == 0 ? nw : warp; c < n; c += nw) {
      C y[MAXR];
      load_col(c, y);
      push_recv(0, c, dot(x, y));
      push_row(y, 0, 0, c);
    }
  }
  cl.sync();
  for (int j = 0; j < k; ++j) {
    const int par = j & 1;
    if (use_gs)
      for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) gs[c] = sum_recv(par, c);
    if (threadIdx.x == blockDim.x - 1) {
      // the reflector of step j from the norm of x and alpha = A[j][j]
      R M = 0, S = 0;
      for (int q = 0; q < cs; ++q) M = fmax(M, pp[par * cs + q].x);
      if (M > 0) {
        const R iM = (R)1 / M;           // (the scales are powers of two: exact)
        for (int q = 0; q < cs; ++q) {
          const C np = pp[par * cs + q];
          const R rq = np.x * iM;
          S += np.y * rq * rq;
        }
      }
      const R xnorm = M * sqrt(S);
      const C alpha = rowb[(size_t)par * n + j];
      const R ar = alpha.x, ai = alpha.y;
      R taur = 0, taui = 0, scr = 0, sci = 0, beta = ar;
      if (!(xnorm == 0 && ai == 0)) {
        // beta = -sign(ar) |(alpha, x)| from scaled terms; alpha - beta
        // scaled by 1 / |beta| (|alpha - beta| >= |beta|), so that nothing
        // overflows or underflows
        const R mx = fmax(fmax(fabs(ar), fabs(ai)), xnorm), imx = (R)1 / mx;
        const R u = ar * imx, w = ai * imx, z = xnorm * imx;
        beta = -copysign(mx * sqrt(u * u + w * w + z * z), ar);
        const R ib = (R)1 / beta, sb = fabs(ib);
        const R dx = (ar - beta) * sb, dy = ai * sb, idd = sb / (dx * dx + dy * dy);
        taur = (beta - ar) * ib;
        taui = -ai * ib;
        scr = dx * idd;
        sci = -dy * idd;
        // (the element type must hold sc too: columns near the bottom of its
        // range leave the column as it is)
        const R smax = sizeof(R) == 4 ? (R)1e37 : (R)1e300;
        if (!(isfinite(taur) && isfinite(taui) && isfinite(scr) && isfinite(sci) && isfinite(beta)) ||
            fabs(scr) > smax || fabs(sci) > smax || beta == (R)0) {
          taur = taui = scr = sci = 0;
          beta = ar;
        }
      }
      const bool act = !(taur == 0 && taui == 0);
      ring[par * 3 + 0] = mkc<C>(taur, taui);
      ring[par * 3 + 1] = mkc<C>(scr, sci);
      ring[par * 3 + 2] = mkc<C>(beta, act ? (R)0 : ai);
      if (Qg) s_tau[j] = mkc<C>(taur, taui);
    }
    __syncthreads();
    const C tj = ring[par * 3 + 0], sc = ring[par * 3 + 1], ctau = mkc<C>(tj.x, -tj.y);
    const bool active = !(tj.x == 0 && tj.y == 0);
    // scale the reflector of step j - 1 (no longer read)
    if (j > 0 && warp == (j - 1) % nw) {
      C x[MAXR];
      load_col(j - 1, x);
      const C scp = ring[(par ^ 1) * 3 + 1], dg = ring[(par ^ 1) * 3 + 2];
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const int g = r0 + lane + 32 * i;
        if (g > j - 1) x[i] = pmul(x[i], scp);
        else if (g == j - 1) x[i] = dg;
      }
      store_col(j - 1, x);
    }
    C v[MAXR];                           // v of step j: x sc below row j, 1 at row j
    load_col(j, v);
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int g = r0 + lane + 32 * i;
      v[i] = g > j ? pmul(v[i], sc) : (g == j ? one : zero);
    }
    auto fac = [&](int c) {
      const C s = use_gs ? gs[c] : sum_recv(par, c);
      return active ? pmul(ctau, padd(rowb[(size_t)par * n + c], pmulc(sc, s))) : zero;
    };
    const bool own = j + 1 < n && warp == (j + 1) % nw;
    C xm[MAXR];                          // column j + 1 after step j, then its rows > j + 1
    C keep_j = zero, keep_j1 = zero;     // (owner) its rows j and j + 1, in the lanes that hold them
    if (j + 1 < n) {
      load_col(j + 1, xm);
      const C f1 = fac(j + 1);
#pragma unroll
      for (int i = 0; i < MAXR; ++i) xm[i] = psub(xm[i], pmul(v[i], f1));
      if (own) {
#pragma unroll
        for (int i = 0; i < MAXR; ++i) {
          const int g = r0 + lane + 32 * i;
          if (g == j) keep_j = xm[i];
          if (g == j + 1) keep_j1 = xm[i];
        }
        if (j + 1 < k) push_row(xm, j + 1, par ^ 1, j + 1);
      }
      mask_below(xm, j + 1);
      if (own && j + 1 < k) push_norm(par ^ 1, norm_part(xm));
      int c = j + 2 + ((warp - (j + 2)) % nw + nw) % nw;
      if constexpr ((sizeof(R) == 4 && MAXR <= 6) || (sizeof(R) == 8 && MAXR <= 2)) {
        // two columns at a time (two independent chains, one reduction
        // tree for both dots: lanes 0-7 end with the first real part, 8-15
        // its imaginary part, 16-31 the second column's)
        for (; c + nw < n; c += 2 * nw) {
          const int c2 = c + nw;
          C y[MAXR], y2[MAXR];
          load_col(c, y);
          load_col(c2, y2);
          const C f = fac(c), f2 = fac(c2);
#pragma unroll
          for (int i = 0; i < MAXR; ++i) {
            y[i] = psub(y[i], pmul(v[i], f));
            y2[i] = psub(y2[i], pmul(v[i], f2));
          }
          store_col(c, y);
          store_col(c2, y2);
          if (j + 1 < k) {
            C d = pmulc(xm[0], y[0]), d2 = pmulc(xm[0], y2[0]);
#pragma unroll
            for (int i = 1; i < MAXR; ++i) {
              d = padd(d, pmulc(xm[i], y[i]));
              d2 = padd(d2, pmulc(xm[i], y2[i]));
            }
            const bool h4 = lane & 16, h3 = lane & 8;
            R a0 = h4 ? d2.x : d.x, a1 = h4 ? d2.y : d.y;     // kept halves
            a0 += __shfl_xor_sync(0xffffffffu, h4 ? d.x : d2.x, 16);
            a1 += __shfl_xor_sync(0xffffffffu, h4 ? d.y : d2.y, 16);
            R b = (h3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, h3 ? a0 : a1, 8);
            b += __shfl_xor_sync(0xffffffffu, b, 4);
            b += __shfl_xor_sync(0xffffffffu, b, 2);
            b += __shfl_xor_sync(0xffffffffu, b, 1);
            const C s1 = mkc<C>(__shfl_sync(0xffffffffu, b, 0), __shfl_sync(0xffffffffu, b, 8));
            const C s2 = mkc<C>(__shfl_sync(0xffffffffu, b, 16), __shfl_sync(0xffffffffu, b, 24));
            push_recv(par ^ 1, c, s1);
            push_recv(par ^ 1, c2, s2);
            push_row(y, j + 1, par ^ 1, c);
            push_row(y2, j + 1, par ^ 1, c2);
          }
        }
      }
      for (; c < n; c += nw) {
        C y[MAXR];
        load_col(c, y);
        const C f = fac(c);
#pragma unroll
        for (int i = 0; i < MAXR; ++i) y[i] = psub(y[i], pmul(v[i], f));
        store_col(c, y);
        if (j + 1 < k) {
          push_recv(par ^ 1, c, dot(xm, y));
          push_row(y, j + 1, par ^ 1, c);
        }
      }
    }
    cl.sync();
    if (own) {                           // column j + 1, rows >= j (rows above are unchanged)
      C* p = A + (size_t)(j + 1) * ld + lane;
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const int g = r0 + lane + 32 * i;
        if (g > j + 1) p[32 * i] = xm[i];
        else if (g == j + 1) p[32 * i] = keep_j1;
        else if (g == j) p[32 * i] = keep_j;
      }
    }
  }
  if (k > 0 && warp == (k - 1) % nw) {   // scale the last reflector
    C x[MAXR];
    load_col(k - 1, x);
    const C scp = ring[((k - 1) & 1) * 3 + 1], dg = ring[((k - 1) & 1) * 3 + 2];
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int g = r0 + lane + 32 * i;
      if (g > k - 1) x[i] = pmul(x[i], scp);
      else if (g == k - 1) x[i] = dg;
    }
    store_col(k - 1, x);
  }
  __syncthreads();

  // R (k x n, upper triangular) from the rows this CTA holds
  if (Rg)
    for (int e = threadIdx.x; e < mr * n; e += blockDim.x) {
      const int t = e / n, c = e % n, g = r0 + t;
      if (g < k) Rg[(long long)g * n + c] = (c >= g) ? A[(size_t)c * ld + t] : zero;
    }
  if (!Qg) return;     // nothing is pushed after the last cluster barrier above

  // ---- Q = H_0 ... H_{k-1} [I; 0] by blocks of NB reflectors, the last
  // block first, in place: H_{b0} ... H_{b1-1} = I - V T V^H (compact WY;
  // T upper triangular, T_jj = tau_j, T_{0:j,j} = -tau_j T_{0:j,0:j}
  // (V^H V)_{0:j,j}), so with Q' the columns >= b1 built so far and e_c the
  // block's own columns,  Q_{:,c} = Q'_{:,c} - V (T (V^H Q'_{:,c})).
  // One cluster exchange per block: every CTA writes its partial V^H Q'
  // and V^H V over its rows into its own shared memory, and after the
  // barrier every CTA sums all CTAs' partials remotely in rank order (the
  // same T and the same products in every CTA).
  constexpr int NB = kQBlock;
  const int W = k + NB;                  // a row of the block buffers: V^H Q' at c < k, V^H V at k + b
  C* Pb = A + L.recv;                    // [2][NB][W]: own partials, by block parity
  C* Sb = Pb + 2 * (size_t)NB * W;       // [NB][W]: cluster sums, then T V^H Q'
  C* Tb = Sb + (size_t)NB * W;           // [NB][NB]
  constexpr int rows_pad = 32 * MAXR;
  const int ngroups = max(1, (int)blockDim.x / rows_pad);
  // V_B[t][a] of the block starting at column b0: reflector b0 + a at local row t
  auto vb = [&](int b0, int a, int t) {
    const int col = b0 + a, g = r0 + t;
    return g > col ? A[(size_t)col * ld + t] : (g == col ? one : zero);
  };
  const int nblk = (k + NB - 1) / NB;
  for (int B = nblk - 1; B >= 0; --B) {
    const int b0 = B * NB, b1 = min(k, b0 + NB), nbB = b1 - b0;
    C* Pw = Pb + (size_t)(B & 1) * NB * W;
    // partials V^H Q' (columns c >= b1): a warp per column, the block's
    // reflectors four at a time in registers
    for (int a0 = 0; a0 < nbB; a0 += 4) {
      C vch[4][MAXR];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int i = 0; i < MAXR; ++i) vch[u][i] = a0 + u < nbB ? vb(b0, a0 + u, lane + 32 * i) : zero;
      for (int c = b1 + ((warp - b1) % nw + nw) % nw; c < k; c += nw) {
        C y[MAXR];
        load_col(c, y);
        R acc[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          C d = pmulc(vch[u][0], y[0]);
#pragma unroll
          for (int i = 1; i < MAXR; ++i) d = padd(d, pmulc(vch[u][i], y[i]));
          acc[2 * u] = d.x;
          acc[2 * u + 1] = d.y;
        }
        // eight sums over the warp, halving the set at every level: lane l
        // ends with sum r = 4 b4 + 2 b3 + b2 of its lane bits
        const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const R send = h4 ? acc[q] : acc[4 + q];
          acc[q] = (h4 ? acc[4 + q] : acc[q]) + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const R send = h3 ? acc[q] : acc[2 + q];
          acc[q] = (h3 ? acc[2 + q] : acc[q]) + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        {
          const R send = h2 ? acc[0] : acc[1];
          acc[0] = (h2 ? acc[1] : acc[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
        if ((lane & 3) == 0) {
          const int r = (h4 ? 4 : 0) + (h3 ? 2 : 0) + (h2 ? 1 : 0), u = r >> 1;
          if (a0 + u < nbB) ((R*)&Pw[(size_t)(a0 + u) * W + c])[r & 1] = acc[0];
        }
      }
    }
    // the block's own columns e_c (c in [b0, b1)): conj(V_B[c][a]) from the
    // CTA that holds row c, zero elsewhere
    for (int e = threadIdx.x; e < nbB * nbB; e += blockDim.x) {
      const int a = e / nbB, c = b0 + e % nbB, t = c - r0;
      const C v = (t >= 0 && t < mr) ? vb(b0, a, t) : zero;
      Pw[(size_t)a * W + c] = mkc<C>(v.x, -v.y);
    }
    // V^H V (a < b) over the slice: a warp per pair
    for (int pr = warp; pr < nbB * nbB; pr += nw) {
      const int a = pr / nbB, b = pr % nbB;
      if (a >= b) continue;
      C x[MAXR], y[MAXR];
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        x[i] = vb(b0, a, lane + 32 * i);
        y[i] = vb(b0, b, lane + 32 * i);
      }
      const C d = dot(x, y);
      if (lane == 0) Pw[(size_t)a * W + k + b] = d;
    }
    cl.sync();
    // cluster sums of the block's partials, read from every CTA in rank order
    for (int e = threadIdx.x; e < nbB * W; e += blockDim.x) {
      const int a = e / W, col = e % W;
      if (col < b0 || (col >= k && (col - k <= a || col - k >= nbB))) continue;
      C sum = zero;
      for (int q0 = 0; q0 < cs; q0 += 8) {
        C vq[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) vq[u] = q0 + u < cs ? cl.map_shared_rank(Pw, q0 + u)[e] : zero;
#pragma unroll
        for (int u = 0; u < 8; ++u) sum = padd(sum, vq[u]);
      }
      Sb[e] = sum;
    }
    __syncthreads();
    if (warp == 0) {                     // T of the block, lane a holds row a
      const int a = lane;
      if (a < NB)
        for (int b = 0; b < NB; ++b) Tb[a * NB + b] = (a == b && a < nbB) ? s_tau[b0 + a] : zero;
      __syncwarp();
      for (int j = 1; j < nbB; ++j) {
        if (a < j) {
          C acc = zero;
          for (int b = a; b < j; ++b) acc = padd(acc, pmul(Tb[a * NB + b], Sb[(size_t)b * W + k + j]));
          const C tj = s_tau[b0 + j];
          Tb[a * NB + j] = mkc<C>(-(tj.x * acc.x - tj.y * acc.y), -(tj.x * acc.y + tj.y * acc.x));
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int c = b0 + threadIdx.x; c < k; c += blockDim.x)   // T V^H Q' in place, rows in ascending order
      for (int a = 0; a < nbB; ++a) {
        C acc = zero;
        for (int b = a; b < nbB; ++b) acc = padd(acc, pmul(Tb[a * NB + b], Sb[(size_t)b * W + c]));
        Sb[(size_t)a * W + c] = acc;
      }
    // every thread takes its row's V_B before the block's columns change
    const int t = threadIdx.x % rows_pad, grp = threadIdx.x / rows_pad;
    C v[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) v[a] = a < nbB ? vb(b0, a, t) : zero;
    __syncthreads();
    if (grp < ngroups) {
      const int g = r0 + t;
      for (int c = b0 + grp; c < k; c += ngroups) {
        C q = c >= b1 ? A[(size_t)c * ld + t] : (g == c ? one : zero);
#pragma unroll
        for (int a = 0; a < NB; ++a)
          if (a < nbB) q = psub(q, pmul(v[a], Sb[(size_t)a * W + c]));
        A[(size_t)c * ld + t] = q;
      }
    }
    __syncthreads();
  }
  cl.sync();                             // no CTA still reads this CTA's partials
  for (int e = threadIdx.x; e < mr * k; e += blockDim.x) {
    const int t = e / k, c = e % k;
    Qg[(long long)(r0 + t) * k + c] = A[(size_t)c * ld + t];
  }
}

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
__host__ __device__ inline size_t panel_smem_pull(int rows, int n) {
  return sizeof(C) * ((size_t)(rows | 1) * n + 4 * (size_t)n + 2 * (size_t)n + 3 * (size_t)n) + 4 * sizeof(double) +
         64;
}

// The pulled form, for panels whose push buffers do not fit: every CTA
// writes its partial sums into a double-buffered slot of its own shared
// memory and, after the cluster barrier, reads every CTA's slot remotely.
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
__global__ void __launch_bounds__(kPanelThreads, 1) k_panel_qr_pull(const C* __restrict__ Ag, int m, int n, int rows,
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

// rows a CTA caches per lane: 32 x MAXR rows per CTA
constexpr int kMaxrF[] = {1, 2, 3, 4, 5, 6, 8};   // complex64
constexpr int kMaxrD[] = {1, 2, 3, 4};            // complex128 (twice the registers per entry)

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

template <typename C, int MAXR>
cudaError_t panel_optin_pull() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_panel_qr_pull<C, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_panel_qr_pull<C, MAXR>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <typename C>
cudaError_t panel_optin() {
  cudaError_t e;
  if ((e = panel_optin_pull<C, 2>()) != cudaSuccess) return e;
  if ((e = panel_optin_pull<C, 4>()) != cudaSuccess) return e;
  if constexpr (sizeof(C) == sizeof(float2))
    if ((e = panel_optin_pull<C, 8>()) != cudaSuccess) return e;
  if ((e = panel_optin_one<C, 1>()) != cudaSuccess) return e;
  if ((e = panel_optin_one<C, 2>()) != cudaSuccess) return e;
  if ((e = panel_optin_one<C, 3>()) != cudaSuccess) return e;
  if ((e = panel_optin_one<C, 4>()) != cudaSuccess) return e;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if ((e = panel_optin_one<C, 5>()) != cudaSuccess) return e;
    if ((e = panel_optin_one<C, 6>()) != cudaSuccess) return e;
    return panel_optin_one<C, 8>();
  }
  return cudaSuccess;
}

struct PanelPlan {
  bool pull = false;
  int maxr = 0, cs = 0, ld = 0, rows = 0;
  bool gs = true;
  size_t bytes = 0;
};

// the first layout that fits: odd column stride (no bank conflicts in the
// row-major copies) with staged sums, even stride, then sums taken in place
template <typename C>
bool panel_fit(int n, int maxr, int cs, bool want_q, PanelPlan& p) {
  for (int v = 0; v < 3; ++v) {
    const PanelLayout L = panel_layout<C>(maxr, n, cs, want_q, v == 0, v < 2);
    if (L.bytes <= (size_t)kPanelSmemMax) {
      p.pull = false;
      p.maxr = maxr;
      p.cs = cs;
      p.ld = L.ld;
      p.rows = 32 * maxr;
      p.gs = v < 2;
      p.bytes = L.bytes;
      return true;
    }
  }
  return false;
}

// the pulled form: rows = ceil(m / cs) a CTA, at most 256 (complex64) or
// 128 (complex128)
template <typename C>
bool panel_fit_pull(int m, int n, int cs, PanelPlan& p) {
  const int rows = (m + cs - 1) / cs;
  const int max_rows = sizeof(C) == sizeof(double2) ? 128 : 256;
  if (rows > max_rows) return false;
  const size_t b = panel_smem_pull<C>(rows, n);
  if (b > (size_t)kPanelSmemMax) return false;
  p.pull = true;
  p.maxr = rows <= 64 ? 2 : (rows <= 128 ? 4 : 8);
  p.cs = cs;
  p.rows = rows;
  p.ld = rows | 1;
  p.bytes = b;
  return true;
}

template <typename C>
void maxr_list(const int*& list, int& nl) {
  if (sizeof(C) == sizeof(float2)) {
    list = kMaxrF;
    nl = (int)(sizeof(kMaxrF) / sizeof(int));
  } else {
    list = kMaxrD;
    nl = (int)(sizeof(kMaxrD) / sizeof(int));
  }
}

// Launch plan of an m x n panel.  A given cluster size takes the fewest rows
// per CTA that cover m; otherwise the fewest rows per CTA whose cluster has
// at most 9 CTAs (complex64: two such clusters share one GPC's SMs, so
// concurrent panels of different streams still place; the complex128 kernel
// is bound by the FP64 rate of its SMs and spreads over up to 16), else up
// to 16 CTAs.  Panels whose push buffers do not fit take the pulled form.
template <typename C>
bool panel_plan(int m, int n, bool want_q, int cluster, PanelPlan& p) {
  if (m < n || n < 1) return false;
  const int* list;
  int nl;
  maxr_list<C>(list, nl);
  if (cluster > 0) {
    if (cluster > kPanelMaxCluster) return false;
    const int need = ((m + cluster - 1) / cluster + 31) / 32;
    for (int a = 0; a < nl; ++a)
      if (list[a] >= need) {
        if (panel_fit<C>(n, list[a], cluster, want_q, p)) return true;
        break;
      }
    return panel_fit_pull<C>(m, n, cluster, p);
  }
  const int pref = sizeof(C) == sizeof(float2) ? 9 : kPanelMaxCluster;
  for (int lim : {pref, kPanelMaxCluster})
    for (int a = 0; a < nl; ++a) {
      const int cs = (m + 32 * list[a] - 1) / (32 * list[a]);
      if (cs <= lim && panel_fit<C>(n, list[a], cs, want_q, p)) return true;
    }
  // pulled: the fewest CTAs that fit, raised to about 256 (complex64) or
  // 64 (complex128) rows a CTA
  for (int cs = 1; cs <= kPanelMaxCluster; ++cs)
    if (panel_fit_pull<C>(m, n, cs, p)) {
      const int target = sizeof(C) == sizeof(float2) ? 256 : 64;
      const int want = std::min(kPanelMaxCluster, std::max(cs, (m + target - 1) / target));
      return panel_fit_pull<C>(m, n, want, p) || panel_fit_pull<C>(m, n, cs, p);
    }
  return false;
}

template <typename C>
int panel_min_cluster(int m, int n, bool want_q) {
  if (m < n || n < 1) return 0;
  const int* list;
  int nl;
  maxr_list<C>(list, nl);
  int best = 0;
  PanelPlan p;
  for (int a = nl - 1; a >= 0; --a) {
    const int cs = (m + 32 * list[a] - 1) / (32 * list[a]);
    if (cs <= kPanelMaxCluster && panel_fit<C>(n, list[a], cs, want_q, p) && (best == 0 || cs < best)) best = cs;
  }
  for (int cs = 1; cs <= kPanelMaxCluster && (best == 0 || cs < best); ++cs)
    if (panel_fit_pull<C>(m, n, cs, p)) {
      best = cs;
      break;
    }
  return best;
}

}  // namespace

cudaError_t init_panel_attributes() {
  cudaError_t e = panel_optin<float2>();
  if (e != cudaSuccess) return e;
  return panel_optin<double2>();
}

int panel_cluster(int m, int n, size_t elem, bool want_q) {
  return elem == sizeof(double2) ? panel_min_cluster<double2>(m, n, want_q) : panel_min_cluster<float2>(m, n, want_q);
}

int panel_cluster_auto(int m, int n, size_t elem, bool want_q) {
  PanelPlan p;
  const bool ok = elem == sizeof(double2) ? panel_plan<double2>(m, n, want_q, 0, p)
                                          : panel_plan<float2>(m, n, want_q, 0, p);
  return ok ? p.cs : 0;
}

template <typename C>
static cudaError_t panel_t(const C* A, int m, int n, C* Q, C* R, int batch, long long stride, cudaStream_t s,
                           int cluster) {
  if (batch < 1 || m < 1 || n < 1) return cudaSuccess;
  PanelPlan p;
  if (!panel_plan<C>(m, n, Q != nullptr, cluster, p)) return cudaErrorInvalidValue;
  cudaError_t e = panel_optin<C>();
  if (e != cudaSuccess) return e;
  KTimerScope timer(KC_ORTH, s, batch * qr_flops(m, n));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.cs * batch, 1, 1);
  cfg.blockDim = dim3(kPanelThreads, 1, 1);
  cfg.dynamicSmemBytes = p.bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = p.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (p.pull) {
    if (p.maxr == 2) return cudaLaunchKernelEx(&cfg, k_panel_qr_pull<C, 2>, A, m, n, p.rows, Q, R, stride);
    if (p.maxr == 4) return cudaLaunchKernelEx(&cfg, k_panel_qr_pull<C, 4>, A, m, n, p.rows, Q, R, stride);
    if constexpr (sizeof(C) == sizeof(float2))
      if (p.maxr == 8) return cudaLaunchKernelEx(&cfg, k_panel_qr_pull<C, 8>, A, m, n, p.rows, Q, R, stride);
    return cudaErrorInvalidValue;
  }
  const int gsf = p.gs ? 1 : 0;
  switch (p.maxr) {
    case 1: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 1>, A, m, n, Q, R, stride, p.ld, gsf);
    case 2: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 2>, A, m, n, Q, R, stride, p.ld, gsf);
    case 3: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 3>, A, m, n, Q, R, stride, p.ld, gsf);
    case 4: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 4>, A, m, n, Q, R, stride, p.ld, gsf);
    default: break;
  }
  if constexpr (sizeof(C) == sizeof(float2)) {
    switch (p.maxr) {
      case 5: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 5>, A, m, n, Q, R, stride, p.ld, gsf);
      case 6: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 6>, A, m, n, Q, R, stride, p.ld, gsf);
      case 8: return cudaLaunchKernelEx(&cfg, k_panel_qr<C, 8>, A, m, n, Q, R, stride, p.ld, gsf);
      default: break;
    }
  }
  return cudaErrorInvalidValue;
}

// ---- panels taller than one cluster holds: row chunks that each fit one,
// their R factors stacked and factorised again, and every chunk's Q
// multiplied by its block of the stack's Q (two-level TSQR):
//   A = [A_0; ...; A_{c-1}],  A_i = Q_i R_i,  [R_0; ...; R_{c-1}] = Qs R,
//   Q = [Q_0 Qs_0; ...; Q_{c-1} Qs_{c-1}]
// Scratch: the chunks' Q (m x n), the stack and its Q (c n x n each).
namespace {
int chunk_count(int m, int n, size_t elem) {
  for (int c = 2; c <= 64; ++c) {
    const int rows = (m + c - 1) / c;
    if (rows < n) break;
    if (panel_cluster(rows, n, elem, true) > 0 && panel_cluster(c * n, n, elem, true) > 0) return c;
  }
  return 0;
}
}  // namespace

size_t panel_chunk_scratch_bytes(int m, int n, size_t elem) {
  if (m < n || n < 1 || panel_cluster(m, n, elem, true) > 0) return 0;
  const int c = chunk_count(m, n, elem);
  if (c == 0) return 0;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  return al(elem * (size_t)m * n) + 2 * al(elem * (size_t)c * n * n);
}

template <typename C>
static cudaError_t panel_chunked_t(const C* A, int m, int n, C* Q, C* R, void* scratch, cudaStream_t s) {
  const int c = chunk_count(m, n, sizeof(C));
  if (c == 0 || !scratch || !Q) return cudaErrorInvalidValue;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  C* Qc = (C*)scratch;
  C* Rs = (C*)((char*)scratch + al(sizeof(C) * (size_t)m * n));
  C* Qs = (C*)((char*)Rs + al(sizeof(C) * (size_t)c * n * n));
  const int rows = (m + c - 1) / c, last = m - (c - 1) * rows;
  cudaError_t e;
  const long long st = (long long)rows * n;
  if ((e = panel_t(A, rows, n, Qc, Rs, c - 1, st, s, 0)) != cudaSuccess) return e;
  if ((e = panel_t(A + (c - 1) * st, last, n, Qc + (c - 1) * st, Rs + (size_t)(c - 1) * n * n, 1, 0, s, 0)) !=
      cudaSuccess)
    return e;
  if ((e = panel_t(Rs, c * n, n, Qs, R, 1, 0, s, 0)) != cudaSuccess) return e;
  const C one = C{1, 0}, zero = C{0, 0};
  if ((e = launch_zgemm('N', 'N', rows, n, n, one, Qc, n, st, Qs, n, (long long)n * n, zero, Q, n, st, c - 1, s)) !=
      cudaSuccess)
    return e;
  return launch_zgemm('N', 'N', last, n, n, one, Qc + (c - 1) * st, n, 0, Qs + (size_t)(c - 1) * n * n, n, 0, zero,
                      Q + (c - 1) * st, n, 0, 1, s);
}

cudaError_t launch_panel_qr_chunked(const float2* A, int m, int n, float2* Q, float2* R, void* scratch,
                                    cudaStream_t s) {
  return panel_chunked_t(A, m, n, Q, R, scratch, s);
}
cudaError_t launch_panel_qr_chunked(const double2* A, int m, int n, double2* Q, double2* R, void* scratch,
                                    cudaStream_t s) {
  return panel_chunked_t(A, m, n, Q, R, scratch, s);
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
