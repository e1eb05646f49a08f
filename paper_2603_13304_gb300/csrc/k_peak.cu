// ALU throughput microbenchmark: independent fused multiply-add chains in
// FP64 or FP32, enough warps per SM to keep the pipe busy.  Measures the
// denominators of the FP64 / FP32 roofline fractions on the device at hand
// (the tensor rates are measured on the tcgen05 GEMM itself).
#include <cuda_runtime.h>

#include "kernels.h"

namespace bbp {

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == (T)-12345.0) out[0] = s;   // never true for the inputs used; keeps the chains live
}

}  // namespace

double fma_peak_flops(bool fp64, int blocks, int iters) {
  return 2.0 * kChains * (double)iters * 256.0 * blocks;
}

cudaError_t launch_fma_peak(bool fp64, int blocks, int iters, void* out, cudaStream_t s) {
  if (fp64) k_fma_peak<double><<<blocks, 256, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
  else k_fma_peak<float><<<blocks, 256, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

}  // namespace bbp
