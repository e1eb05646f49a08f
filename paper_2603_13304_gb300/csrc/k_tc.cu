// Tensor-core GEMM for the absorb contraction (K2, Sec. 1.1.3 / Sec. 2.3.3):
// tcgen05.mma with the accumulator in TMEM, operands staged into shared
// memory by TMA (128-byte swizzle, K-major), a 4-stage mbarrier pipeline.
//
// Real GEMM  C (M x N, fp32, row-major) = alpha * A (M x K) * B (K x N)
// with A given K-major (row-major M x K) and B given as B^T (row-major
// N x K).  Operands are TF32 (kind::tf32, 32-bit storage) or BF16
// (kind::f16).  One CTA of 128 threads computes a 128 x BN tile:
//   warp 0, one lane : TMA producer
//   warp 1, one lane : MMA issuer (tcgen05.mma, tcgen05.commit -> mbarrier)
//   warps 0-3        : epilogue, TMEM lanes 32w..32w+31 -> rows of C
// Every mbarrier wait is bounded by the global timer; on expiry the kernel
// records an error, drains its own TMA copies and MMAs (bounded), releases
// TMEM and returns.
//
// The complex contraction R[a] = X^T S[a] (batched over a) runs as one real
// GEMM: X^T and S are scaled by a power of two (largest magnitude about 1)
// and split into limbs of the operand type, and the K dimension concatenates
// segments that pair a limb of A with a limb of B:
//   A = [ Re a, -Im a ]  (rows q),  [ Im a, Re a ]  (rows Q + q)  per segment
//   B = [ Re b ; Im b ]                                           per segment
// TF32: limbs hi, lo and the segments hi*hi, hi*lo, lo*hi; BF16 (8 bits a
// limb): limbs h, m, l and the segments hh, hm, mh, hl, mm, lh.  Both
// accumulate in FP32 in one pass to about FP32 accuracy.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <initializer_list>
#include <map>
#include <mutex>
#include <set>
#include <vector>

#include "kernels.h"

namespace bbp {

namespace {

constexpr int kBM = 128;
// pipeline depth: one stage holds 4 MMAs of 128 x BN x (32 bytes of K), a
// fraction of a microsecond of tensor work, so enough stages must be in
// flight to cover the TMA latency from L2: 4 at BN = 256, 6 at BN = 128, 8
// at BN = 64 (about 192 KB of shared memory each)
template <int BN> __host__ __device__ constexpr int stages_of() { return BN >= 256 ? 4 : (BN >= 128 ? 6 : 8); }
// tile order: groups of group_m M tiles sweep the N tiles together, so that
// a wave of CTAs reuses its A tiles from L2 instead of streaming all of B
// (group_m is a launch parameter, picked per shape by the autotuner)
constexpr int kGroupMDefault = 16;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// Wait for the phase of the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = saddr(bar);
  unsigned long long t0 = 0;
  for (long long it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = gtimer();
    else if (gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          saddr(dst)),
      "l"(map), "r"(saddr(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout TMA writes for a 128-byte-wide box).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t a) {
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

template <bool kBF16>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  if constexpr (kBF16)
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(
            tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Instruction descriptor: FP32 accumulator, A/B K-major, M = 128, N = BN.
template <bool kBF16, int BN>
__host__ __device__ constexpr uint32_t idesc_of() {
  const uint32_t fmt = kBF16 ? 1u : 2u;   // BF16 (kind::f16) or TF32 (kind::tf32)
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

template <bool kBF16, int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, float* __restrict__ C,
              int M, int N, int K, long long ldc, float alpha, int* err, int group_m) {
  constexpr int kEs = kBF16 ? 2 : 4;
  constexpr int kBKe = 128 / kEs;               // K elements per stage (one 128-byte row)
  constexpr int kUmmaK = 32 / kEs;              // K elements per tcgen05.mma
  constexpr int kABytes = kBM * 128, kBBytes = BN * 128, kStageBytes = kABytes + kBBytes;
  constexpr int kStages = stages_of<BN>();
  constexpr uint32_t kIdesc = idesc_of<kBF16, BN>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterisation of the linear block index
  const int tiles_n = gridDim.x, tiles_m = gridDim.y;
  const int pid = blockIdx.y * tiles_n + blockIdx.x;
  const int group = pid / (group_m * tiles_n), first_m = group * group_m;
  const int gm = min(group_m, tiles_m - first_m);
  const int in_group = pid - group * group_m * tiles_n;
  const int tm = first_m + in_group % gm, tn = in_group / gm;
  const int n0 = tn * BN, m0 = tm * kBM;
  const int kt = (K + kBKe - 1) / kBKe;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                 "r"((uint32_t)BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int k = 0; k < kt; ++k) {
      const int s = k % kStages;
      const uint32_t ph = (uint32_t)(k / kStages) & 1u;
      if (k >= kStages && !mbar_wait(&empty[s], ph ^ 1u)) {
        s_fail = 1;
        break;
      }
      mbar_expect_tx(&full[s], kStageBytes);
      tma_load_2d(base + s * kStageBytes, &tA, &full[s], k * kBKe, m0);
      tma_load_2d(base + s * kStageBytes + kABytes, &tB, &full[s], k * kBKe, n0);
      ++issued;
    }
    // no copy of ours may still be in flight when the CTA exits
    for (int k = issued - kStages < 0 ? 0 : issued - kStages; k < issued; ++k)
      if (!mbar_wait(&full[k % kStages], (uint32_t)(k / kStages) & 1u)) s_fail = 1;
  } else if (warp == 1 && lane == 0) {
    for (int k = 0; k < kt; ++k) {
      const int s = k % kStages;
      if (!mbar_wait(&full[s], (uint32_t)(k / kStages) & 1u)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = saddr(base + s * kStageBytes), b = a + kABytes;
#pragma unroll
      for (int kk = 0; kk < kBKe / kUmmaK; ++kk)
        umma<kBF16>(tmem, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), kIdesc, (k | kk) != 0);
      umma_commit(&empty[s]);
    }
    umma_commit(&done);   // arrives once every MMA issued above has completed
  }
  __syncwarp();
  if (!mbar_wait(&done, 0)) s_fail = 1;
  __syncwarp();   // tcgen05.ld below is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const int row = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (row < M && kt > 0) {
      float* out = C + (long long)row * ldc + n0 + c0;
      const int lim = N - n0 - c0;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < lim) out[j] = alpha * __uint_as_float(v[j]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN));
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ------------------------------------------------------------ host: TMA maps

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// rows x cols row-major operand (cols = K, contiguous), box = box_rows x 128 bytes
bool make_map(CUtensorMap* m, const void* ptr, bool bf16, int rows, int cols, long long ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN> constexpr int tc_smem() { return stages_of<BN>() * (kBM + BN) * 128 + 1024; }

// Dynamic shared memory opt-in, once per kernel and device.
template <bool kBF16, int BN>
cudaError_t tc_optin() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_tc_gemm<kBF16, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<BN>());
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <bool kBF16, int BN>
cudaError_t tc_launch(const void* A, long long lda, const void* Bt, long long ldb, float* C, long long ldc, int M, int N,
                      int K, float alpha, int* err, cudaStream_t s, double algo_flops, int group_m) {
  constexpr int smem = tc_smem<BN>();
  cudaError_t attr_err = tc_optin<kBF16, BN>();
  if (attr_err != cudaSuccess) return attr_err;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, kBF16, M, K, lda, kBM) || !make_map(&tb, Bt, kBF16, N, K, ldb, BN))
    return cudaErrorInvalidValue;
  dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM);
  KTimerScope timer(KC_TC, s, algo_flops > 0 ? algo_flops : 2.0 * M * N * K);
  k_tc_gemm<kBF16, BN><<<grid, 128, smem, s>>>(ta, tb, C, M, N, K, ldc, alpha, err, group_m < 1 ? 1 : group_m);
  return cudaGetLastError();
}

// ----------------------------------------------------- complex <-> real packing

template <bool kBF16> struct Op;
template <> struct Op<false> {
  using T = float;
  static __device__ __forceinline__ float round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
  static __device__ __forceinline__ float store(float x) { return x; }
};
template <> struct Op<true> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
  static __device__ __forceinline__ __nv_bfloat16 store(float x) { return __float2bfloat16_rn(x); }
};

template <typename C> __device__ __forceinline__ double2 ld_c(const C* p, long long i);
template <> __device__ __forceinline__ double2 ld_c(const double2* p, long long i) { return p[i]; }
template <> __device__ __forceinline__ double2 ld_c(const float2* p, long long i) {
  float2 v = p[i];
  return make_double2(v.x, v.y);
}

// largest |Re|, |Im| of n complex entries -> *out (as the bits of a
// non-negative float, so atomicMax on int orders them)
template <typename C>
__global__ void k_absmax(const C* __restrict__ x, long long n, int* out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 v = ld_c(x, i);
    m = fmaxf(m, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_int(m));
}

// power-of-two scale bringing the largest magnitude near 1
__device__ __forceinline__ float pow2_scale(const int* amax) {
  const float m = __int_as_float(*amax);
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  return exp2f(-(float)ilogbf(m));
}

// Split of a (scaled) value into limbs of the operand type: TF32 keeps two
// limbs (hi, lo) and the three products hi*hi + hi*lo + lo*hi; BF16, with 8
// significant bits a limb, keeps three (h, m, l) and the six products of
// order up to 2^-16, hh + hm + mh + hl + mm + lh, so that both reach about
// FP32 accuracy.  Segment s of the K dimension pairs limb kLimbA[s] of A with
// limb kLimbB[s] of B.
template <bool kBF16> struct Split;
template <> struct Split<false> {
  static constexpr int kSegs = 3;
  static __device__ __forceinline__ int limb_a(int s) { return s == 2 ? 1 : 0; }   // hi hi lo
  static __device__ __forceinline__ int limb_b(int s) { return s == 1 ? 1 : 0; }   // hi lo hi
};
template <> struct Split<true> {
  static constexpr int kSegs = 6;
  static __device__ __forceinline__ int limb_a(int s) { return (0x210100 >> (4 * s)) & 15; }   // h h m h m l
  static __device__ __forceinline__ int limb_b(int s) { return (0x012010 >> (4 * s)) & 15; }   // h m h l m h
};

template <bool kBF16>
__device__ __forceinline__ float limb(float x, int which) {
  using O = Op<kBF16>;
  const float h = O::round(x);
  if (which == 0) return h;
  const float r1 = x - h, m = O::round(r1);
  if (which == 1) return m;
  return O::round(r1 - m);
}

// A operand from X (P x Q complex, row-major): rows q and Q + q, K index
// laid out [segment] x [Re/Im block of P]; row stride lda >= 2 kSegs P.
template <bool kBF16, typename C>
__global__ void k_pack_a(const C* __restrict__ X, int P, int Q, const int* amax, typename Op<kBF16>::T* A, long long lda) {
  using O = Op<kBF16>;
  using S = Split<kBF16>;
  const float sc = pow2_scale(amax);
  const long long tot = (long long)Q * lda;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / lda), kk = (int)(e % lda);
    float v0 = 0.f, v1 = 0.f;   // rows q (real part) and Q + q (imaginary part)
    if (kk < 2 * S::kSegs * P) {
      const int blk = kk / (2 * P), rem = kk % (2 * P), p = rem % P;
      const bool im_half = rem >= P;
      double2 x = ld_c(X, (long long)p * Q + q);
      const int w = S::limb_a(blk);
      const float xr = limb<kBF16>((float)x.x * sc, w), xi = limb<kBF16>((float)x.y * sc, w);
      // row q: [Re, -Im]; row Q + q: [Im, Re]
      v0 = im_half ? -xi : xr;
      v1 = im_half ? xr : xi;
    }
    A[(long long)q * lda + kk] = O::store(v0);
    A[(long long)(Q + q) * lda + kk] = O::store(v1);
  }
}

// B^T operand from S (l x P x r complex): row n = a * r + c, K index laid
// out [segment] x [Re/Im block of P]; row stride ldb >= 2 kSegs P.
template <bool kBF16, typename C>
__global__ void k_pack_b(const C* __restrict__ S, int l, int P, int r, const int* amax, typename Op<kBF16>::T* B,
                         long long ldb) {
  using O = Op<kBF16>;
  using Sp = Split<kBF16>;
  const float sc = pow2_scale(amax);
  const long long N = (long long)l * r;
  const long long tot = N * ldb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long n = e / ldb;
    const int kk = (int)(e % ldb);
    float v = 0.f;
    if (kk < 2 * Sp::kSegs * P) {
      const int blk = kk / (2 * P), rem = kk % (2 * P), p = rem % P;
      const bool im_half = rem >= P;
      const int a = (int)(n / r), c = (int)(n % r);
      double2 x = ld_c(S, ((long long)a * P + p) * r + c);
      v = limb<kBF16>((float)(im_half ? x.y : x.x) * sc, Sp::limb_b(blk));
    }
    B[e] = O::store(v);
  }
}

template <typename C> __device__ __forceinline__ C mk(double re, double im);
template <> __device__ __forceinline__ double2 mk(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 mk(double re, double im) { return make_float2((float)re, (float)im); }

// R[a][q][c] = (Cr[q][a r + c] + i Ci[q][a r + c]) / (scale_A scale_B)
template <typename C>
__global__ void k_unpack(const float* __restrict__ Cm, long long ldc, int Q, int l, int r, const int* amax_a,
                         const int* amax_b, C* R) {
  const double inv = 1.0 / ((double)pow2_scale(amax_a) * (double)pow2_scale(amax_b));
  const long long tot = (long long)l * Q * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % r);
    const long long t = e / r;
    const int q = (int)(t % Q), a = (int)(t / Q);
    const long long n = (long long)a * r + c;
    R[e] = mk<C>(Cm[(long long)q * ldc + n] * inv, Cm[(long long)(Q + q) * ldc + n] * inv);
  }
}

// ------------------------------------------- general complex GEMM operands
//
// C (M x N complex) = op(A) (M x K) op(B) (K x N) as one real GEMM whose
// output is C itself, read as an M x 2N real matrix (interleaved re, im):
//   A'' (M x 6K):  [ hi | hi | lo ] of [re a_0, im a_0, re a_1, im a_1, ...]
//   B'' (2N x 6K): row 2j   = [ hi | lo | hi ] of [ re b_0j, -im b_0j, ... ]
//                  row 2j+1 = [ hi | lo | hi ] of [ im b_0j,  re b_0j, ... ]
// so that the K sum pairs a_k with b_kj and hi*hi + hi*lo + lo*hi
// accumulates in FP32.  No scaling: TF32 and BF16 keep FP32's exponent
// range.  Rows are padded to ldK (a multiple of 32) with zeros.

template <typename C> __device__ __forceinline__ float2 ld_f2(const C* p, long long i);
template <> __device__ __forceinline__ float2 ld_f2(const float2* p, long long i) { return p[i]; }
template <> __device__ __forceinline__ float2 ld_f2(const double2* p, long long i) {
  const double2 v = p[i];
  return make_float2((float)v.x, (float)v.y);
}

template <bool kBF16>
__device__ __forceinline__ float split_part(float v, int seg_is_lo) {
  using O = Op<kBF16>;
  const float h = O::round(v);
  return seg_is_lo ? O::round(v - h) : h;
}

// A'' from op(A) = A (op 'N', A row-major M x K, row stride lda): coalesced
template <bool kBF16, typename C>
__global__ void k_zpack_an(const C* __restrict__ A, long long lda, int M, int K, typename Op<kBF16>::T* out,
                           long long ldK) {
  using O = Op<kBF16>;
  const long long tot = (long long)M * ldK;
  const int K2 = 2 * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ldK), kk = (int)(e % ldK);
    float v = 0.f;
    if (kk < 3 * K2) {
      const int seg = kk / K2, rem = kk % K2;
      const float2 z = ld_f2(A, (long long)i * lda + (rem >> 1));
      v = split_part<kBF16>((rem & 1) ? z.y : z.x, seg == 2);
    }
    out[e] = O::store(v);
  }
}

// A'' from op(A) = A^T or A^H (A row-major K x M, row stride lda): a 32 x 32
// tile of A is read along its rows and written transposed.
template <bool kBF16, typename C>
__global__ void __launch_bounds__(256) k_zpack_at(const C* __restrict__ A, long long lda, bool conj, int M, int K,
                                                  typename Op<kBF16>::T* out, long long ldK) {
  using O = Op<kBF16>;
  __shared__ float2 tile[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, i = i0 + tx;
    float2 z = make_float2(0.f, 0.f);
    if (k < K && i < M) z = ld_f2(A, (long long)k * lda + i);
    if (conj) z.y = -z.y;
    tile[r][tx] = z;                      // tile[k - k0][i - i0]
  }
  __syncthreads();
  const int K2 = 2 * K;
  // each output row i gets 3 segments x 64 reals from this tile
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    if (i >= M) continue;
    for (int q = tx; q < 3 * 64; q += 32) {
      const int seg = q / 64, w = q % 64, k = k0 + (w >> 1);
      if (k >= K) continue;
      const float2 z = tile[w >> 1][r];
      out[(long long)i * ldK + (long long)seg * K2 + 2 * k + (w & 1)] =
          O::store(split_part<kBF16>((w & 1) ? z.y : z.x, seg == 2));
    }
  }
}

__global__ void k_zero_pad(float* out, int rows, long long ldK, long long from) {
  const long long w = ldK - from;
  const long long tot = (long long)rows * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    out[(e / w) * ldK + from + e % w] = 0.f;
}
__global__ void k_zero_pad_bf(__nv_bfloat16* out, int rows, long long ldK, long long from) {
  const long long w = ldK - from;
  const long long tot = (long long)rows * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x)
    out[(e / w) * ldK + from + e % w] = __float2bfloat16_rn(0.f);
}

// B'' (2N x ldK) from op(B) (K x N): 'N' B row-major K x N (stride ldb),
// 'T' / 'C' B row-major N x K.
template <bool kBF16, typename C>
__global__ void k_zpack_b(const C* __restrict__ B, long long ldb, char op, int K, int N, typename Op<kBF16>::T* out,
                          long long ldK) {
  using O = Op<kBF16>;
  const long long tot = 2LL * N * ldK;
  const int K2 = 2 * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / ldK;
    const int kk = (int)(e % ldK);
    float v = 0.f;
    if (kk < 3 * K2) {
      const int j = (int)(row >> 1), t = (int)(row & 1);
      const int seg = kk / K2, rem = kk % K2, k = rem >> 1, u = rem & 1;
      float2 z = (op == 'N') ? ld_f2(B, (long long)k * ldb + j) : ld_f2(B, (long long)j * ldb + k);
      if (op == 'C') z.y = -z.y;
      // (t, u): (0,0) re, (0,1) -im, (1,0) im, (1,1) re
      const float x = (t == u) ? z.x : (t == 0 ? -z.y : z.y);
      v = split_part<kBF16>(x, seg == 1);
    }
    out[e] = O::store(v);
  }
}

int grid_of(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ------------------------------------------------------------------ public

cudaError_t init_tc_attributes() {
  cudaError_t e;
  if ((e = tc_optin<false, 64>()) != cudaSuccess) return e;
  if ((e = tc_optin<false, 128>()) != cudaSuccess) return e;
  if ((e = tc_optin<false, 256>()) != cudaSuccess) return e;
  if ((e = tc_optin<true, 64>()) != cudaSuccess) return e;
  if ((e = tc_optin<true, 128>()) != cudaSuccess) return e;
  return tc_optin<true, 256>();
}

cudaError_t launch_tc_gemm_tile(bool bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C,
                                long long ldc, int M, int N, int K, float alpha, int* err, cudaStream_t s, int bn,
                                int group_m, double algo_flops) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int es = bf16 ? 2 : 4;
  if ((lda * es) % 16 || (ldb * es) % 16 || ((uintptr_t)A & 15) || ((uintptr_t)Bt & 15)) return cudaErrorInvalidValue;
  switch (bn) {
    case 64:
      return bf16 ? tc_launch<true, 64>(A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, algo_flops, group_m)
                  : tc_launch<false, 64>(A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, algo_flops, group_m);
    case 128:
      return bf16 ? tc_launch<true, 128>(A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, algo_flops, group_m)
                  : tc_launch<false, 128>(A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, algo_flops, group_m);
    case 256:
      return bf16 ? tc_launch<true, 256>(A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, algo_flops, group_m)
                  : tc_launch<false, 256>(A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, algo_flops, group_m);
    default:
      return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------ autotuner
//
// The tile of a launch (BN, the width of a CTA's output tile, and group_m,
// the M tiles a wave sweeps together) is looked up by the exact GEMM shape
// (precision, M, N, K); shapes not in the table take the size rule (BN 128
// above N = 64, else 64; group_m 16).  While recording is on, unknown shapes
// are collected; tc_autotune times every candidate tile of each collected
// shape on scratch operands (CUDA events, outside any capture) and keeps
// the fastest.  The table can be written to and read from a text cache.
namespace {

struct TcKey {
  int bf16, M, N, K;
  bool operator<(const TcKey& o) const {
    if (bf16 != o.bf16) return bf16 < o.bf16;
    if (M != o.M) return M < o.M;
    if (N != o.N) return N < o.N;
    return K < o.K;
  }
};
struct TcTile {
  int bn = 0, group_m = kGroupMDefault;
  float us = 0.f;
};
std::mutex g_tune_mu;
std::map<TcKey, TcTile> g_tiles;
std::set<TcKey> g_pending;
std::atomic<bool> g_recording{false};
std::atomic<unsigned long long> g_tune_gen{0};

TcTile rule_tile(int N) {
  TcTile t;
  t.bn = N > 64 ? 128 : 64;
  return t;
}

bool write_cache(const char* path) {
  FILE* f = std::fopen(path, "w");
  if (!f) return false;
  std::fprintf(f, "# bbp tensor-core GEMM tiles: tc bf16 M N K bn group_m microseconds\n");
  for (const auto& kv : g_tiles)
    std::fprintf(f, "tc %d %d %d %d %d %d %.3f\n", kv.first.bf16, kv.first.M, kv.first.N, kv.first.K, kv.second.bn,
                 kv.second.group_m, kv.second.us);
  return std::fclose(f) == 0;
}

}  // namespace

unsigned long long tc_tune_generation() { return g_tune_gen.load(); }

void tc_autotune_record(bool on) { g_recording.store(on); }

void tc_autotune_info(int* entries, int* pending) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (entries) *entries = (int)g_tiles.size();
  if (pending) *pending = (int)g_pending.size();
}

void tc_autotune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tiles.clear();
  g_pending.clear();
  ++g_tune_gen;
}

cudaError_t tc_autotune(const char* cache_path, int* tuned) {
  if (tuned) *tuned = 0;
  std::vector<TcKey> todo;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const TcKey& k : g_pending)
      if (!g_tiles.count(k)) todo.push_back(k);
    g_pending.clear();
  }
  cudaError_t e = init_tc_attributes();
  if (e != cudaSuccess) return e;
  cudaStream_t s = nullptr;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int* err = nullptr;
  cudaMalloc(&err, sizeof(int));
  int n_done = 0;
  for (const TcKey& k : todo) {
    const size_t es = k.bf16 ? 2 : 4;
    const long long ld = ((long long)k.K + 31) / 32 * 32;
    void *A = nullptr, *B = nullptr;
    float* C = nullptr;
    if (cudaMalloc(&A, (size_t)k.M * ld * es) != cudaSuccess || cudaMalloc(&B, (size_t)k.N * ld * es) != cudaSuccess ||
        cudaMalloc(&C, sizeof(float) * (size_t)k.M * k.N) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(A);
      cudaFree(B);
      cudaFree(C);
      continue;   // no scratch for this shape: it keeps the size rule
    }
    cudaMemsetAsync(A, 0, (size_t)k.M * ld * es, s);
    cudaMemsetAsync(B, 0, (size_t)k.N * ld * es, s);
    cudaMemsetAsync(err, 0, sizeof(int), s);
    TcTile best;
    best.us = 1e30f;
    const int tiles_m = (k.M + kBM - 1) / kBM;
    for (int bn : {64, 128, 256}) {
      if (bn == 256 && k.N <= 128) continue;
      if (bn == 64 && k.N > 1024) continue;
      for (int gm : {1, 8, 16}) {
        // groups of at least tiles_m M tiles all give one group (the same order)
        if ((gm == 16 && tiles_m <= 8) || (gm == 8 && tiles_m <= 1)) continue;
        if (launch_tc_gemm_tile(k.bf16 != 0, A, ld, B, ld, C, k.N, k.M, k.N, k.K, 1.f, err, s, bn, gm, 0.0) !=
            cudaSuccess)
          continue;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch_tc_gemm_tile(k.bf16 != 0, A, ld, B, ld, C, k.N, k.M, k.N, k.K, 1.f, err, s, bn, gm, 0.0);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = 1e3f * ms / 3.f;
        if (us < best.us) {
          best.bn = bn;
          best.group_m = gm;
          best.us = us;
        }
      }
    }
    cudaStreamSynchronize(s);
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    if (best.bn) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tiles[k] = best;
      ++n_done;
    }
  }
  int h_err = 0;
  cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (n_done) ++g_tune_gen;
  if (tuned) *tuned = n_done;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (h_err) return cudaErrorLaunchTimeout;
  if (cache_path && *cache_path) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!write_cache(cache_path)) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

int tc_autotune_load(const char* cache_path) {
  FILE* f = std::fopen(cache_path, "r");
  if (!f) return -1;
  char line[256];
  int n = 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (std::fgets(line, sizeof(line), f)) {
    TcKey k;
    TcTile t;
    if (std::sscanf(line, "tc %d %d %d %d %d %d %f", &k.bf16, &k.M, &k.N, &k.K, &t.bn, &t.group_m, &t.us) != 7) continue;
    if ((t.bn != 64 && t.bn != 128 && t.bn != 256) || t.group_m < 1 || k.M < 1 || k.N < 1 || k.K < 1) continue;
    g_tiles[k] = t;
    ++n;
  }
  std::fclose(f);
  if (n) ++g_tune_gen;
  return n;
}

cudaError_t launch_tc_gemm(bool bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C,
                           long long ldc, int M, int N, int K, float alpha, int* err, cudaStream_t s,
                           double algo_flops) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  TcTile t = rule_tile(N);
  {
    const TcKey key{bf16 ? 1 : 0, M, N, K};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tiles.find(key);
    if (it != g_tiles.end()) t = it->second;
    else if (g_recording.load(std::memory_order_relaxed)) g_pending.insert(key);
  }
  return launch_tc_gemm_tile(bf16, A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err, s, t.bn, t.group_m, algo_flops);
}

long long tc_ld(int P) { return ((6LL * P + 31) / 32) * 32; }
// K extent of the absorb operands: 2 P reals a segment, 3 segments (TF32) or 6 (BF16)
long long tc_absorb_ld(bool bf16, int P) { return ((2LL * (bf16 ? 6 : 3) * P + 31) / 32) * 32; }

// ------------------------------------------------ general complex GEMM (c64)

size_t tc_zpack_bytes(bool bf16, int rows, int K) {
  const size_t es = bf16 ? 2 : 4;
  return ((size_t)rows * (size_t)tc_ld(K) * es + 255) / 256 * 256;
}

template <bool kBF16, typename C>
static cudaError_t zpack_a_t(char opA, int M, int K, const C* A, long long lda, void* out, cudaStream_t s) {
  using T = typename Op<kBF16>::T;
  const long long ldK = tc_ld(K);
  if (opA == 'N') {
    k_zpack_an<kBF16, C><<<grid_of((long long)M * ldK), 256, 0, s>>>(A, lda, M, K, (T*)out, ldK);
  } else {
    dim3 g((M + 31) / 32, (K + 31) / 32);
    k_zpack_at<kBF16, C><<<g, 256, 0, s>>>(A, lda, opA == 'C', M, K, (T*)out, ldK);
    if (ldK > 6LL * K) {
      if (kBF16) k_zero_pad_bf<<<grid_of((long long)M * (ldK - 6LL * K)), 256, 0, s>>>((__nv_bfloat16*)out, M, ldK, 6LL * K);
      else k_zero_pad<<<grid_of((long long)M * (ldK - 6LL * K)), 256, 0, s>>>((float*)out, M, ldK, 6LL * K);
    }
  }
  return cudaGetLastError();
}

cudaError_t tc_zpack_a(bool bf16, char opA, int M, int K, const float2* A, long long lda, void* out, cudaStream_t s) {
  return bf16 ? zpack_a_t<true>(opA, M, K, A, lda, out, s) : zpack_a_t<false>(opA, M, K, A, lda, out, s);
}

cudaError_t tc_zpack_b(bool bf16, char opB, int K, int N, const float2* B, long long ldb, void* out, cudaStream_t s) {
  const long long ldK = tc_ld(K);
  if (bf16) k_zpack_b<true, float2><<<grid_of(2LL * N * ldK), 256, 0, s>>>(B, ldb, opB, K, N, (__nv_bfloat16*)out, ldK);
  else k_zpack_b<false, float2><<<grid_of(2LL * N * ldK), 256, 0, s>>>(B, ldb, opB, K, N, (float*)out, ldK);
  return cudaGetLastError();
}

cudaError_t tc_zgemm_packed(bool bf16, int M, int N, int K, const void* Ap, const void* Bp, float2* Cm, long long ldc,
                            int* err, cudaStream_t s) {
  const long long ldK = tc_ld(K);
  return launch_tc_gemm(bf16, Ap, ldK, Bp, ldK, (float*)Cm, 2 * ldc, M, 2 * N, (int)ldK, 1.0f, err, s,
                        8.0 * M * N * (double)K);
}

size_t tc_absorb_bytes(bool bf16, int P, int Q, int l, int r) {
  const size_t es = bf16 ? 2 : 4;
  const size_t ld = (size_t)tc_absorb_ld(bf16, P);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  return al(2 * (size_t)Q * ld * es) + al((size_t)l * r * ld * es) + al(sizeof(float) * 2 * (size_t)Q * l * r) + 256;
}

template <typename C>
static cudaError_t tc_absorb_t(bool bf16, const C* X, int P, int Q, const C* S, int l, int r, C* R, void* work,
                               int* err, cudaStream_t s) {
  const size_t es = bf16 ? 2 : 4;
  const long long ld = tc_absorb_ld(bf16, P);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char* p = (char*)work;
  void* A = p;
  p += al(2 * (size_t)Q * ld * es);
  void* B = p;
  p += al((size_t)l * r * ld * es);
  float* Cm = (float*)p;
  p += al(sizeof(float) * 2 * (size_t)Q * l * r);
  int* amax = (int*)p;   // [0] X, [1] S
  cudaError_t e;
  if ((e = cudaMemsetAsync(amax, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
  k_absmax<C><<<grid_of((long long)P * Q), 256, 0, s>>>(X, (long long)P * Q, amax);
  k_absmax<C><<<grid_of((long long)l * P * r), 256, 0, s>>>(S, (long long)l * P * r, amax + 1);
  if (bf16) {
    k_pack_a<true, C><<<grid_of((long long)Q * ld), 256, 0, s>>>(X, P, Q, amax, (__nv_bfloat16*)A, ld);
    k_pack_b<true, C><<<grid_of((long long)l * r * ld), 256, 0, s>>>(S, l, P, r, amax + 1, (__nv_bfloat16*)B, ld);
  } else {
    k_pack_a<false, C><<<grid_of((long long)Q * ld), 256, 0, s>>>(X, P, Q, amax, (float*)A, ld);
    k_pack_b<false, C><<<grid_of((long long)l * r * ld), 256, 0, s>>>(S, l, P, r, amax + 1, (float*)B, ld);
  }
  const int N = l * r;
  if ((e = launch_tc_gemm(bf16, A, ld, B, ld, Cm, N, 2 * Q, N, (int)ld, 1.0f, err, s, 8.0 * Q * N * (double)P)) !=
      cudaSuccess)
    return e;
  k_unpack<C><<<grid_of((long long)l * Q * r), 256, 0, s>>>(Cm, N, Q, l, r, amax, amax + 1, R);
  return cudaGetLastError();
}

cudaError_t launch_tc_absorb(bool bf16, const double2* X, int P, int Q, const double2* S, int l, int r, double2* R,
                             void* work, int* err, cudaStream_t s) {
  return tc_absorb_t(bf16, X, P, Q, S, l, r, R, work, err, s);
}
cudaError_t launch_tc_absorb(bool bf16, const float2* X, int P, int Q, const float2* S, int l, int r, float2* R,
                             void* work, int* err, cudaStream_t s) {
  return tc_absorb_t(bf16, X, P, Q, S, l, r, R, work, err, s);
}

}  // namespace bbp
