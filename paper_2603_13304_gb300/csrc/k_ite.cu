// Small kernels of the ITE bond update (Ch. 3, "ITE update step"): the
// problem sizes are those of one bond (d D^4 entries a site tensor, the
// bond's environment over its six outer legs), so these are plain
// one-thread-per-entry or one-CTA kernels; the contractions themselves run on
// the complex GEMM.
#include <cuda_runtime.h>

#include "kernels.h"

namespace bbp {

namespace {

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

__global__ void k_strided_copy(const double2* __restrict__ src, double2* __restrict__ dst, StridedView v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < v.total;
       e += (long long)gridDim.x * blockDim.x) {
    long long rem = e, so = 0, dof = 0;
    for (int q = v.rank - 1; q >= 0; --q) {
      const long long c = rem % v.dims[q];
      rem /= v.dims[q];
      so += c * v.sstr[q];
      dof += c * v.dstr[q];
    }
    dst[dof] = src[so];
  }
}

// W[i, :] *= 1 / s2[i] with s2[i] = |Rem[i, :]|^2 (the square of the i-th
// singular value), 0 where s2[i] <= rcond^2 max s2.  One CTA.
__global__ void k_pinv_rows(double2* W, const double2* __restrict__ Rem, int n, int ncols, double rcond) {
  extern __shared__ double s2[];
  __shared__ double smax;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
      const double2 v = Rem[(long long)i * n + j];
      acc += v.x * v.x + v.y * v.y;
    }
    s2[i] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, s2[i]);
    smax = m;
  }
  __syncthreads();
  const double cut = rcond * rcond * smax;
  for (int e = threadIdx.x; e < n * ncols; e += blockDim.x) {
    const int i = e / ncols;
    const double f = s2[i] > cut ? 1.0 / s2[i] : 0.0;
    W[e] = make_double2(W[e].x * f, W[e].y * f);
  }
}

// out = Re sum_e T[e] conj(X[e]).  One CTA.
__global__ void k_quad_form(const double2* __restrict__ T, const double2* __restrict__ X, long long n, double* out) {
  __shared__ double part[256];
  double acc = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) acc += cmulc(T[e], X[e]).x;
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

// A /= max |A| (A unchanged when it is zero).  One CTA.
__global__ void k_scale_absmax(double2* A, long long n) {
  __shared__ double part[256];
  double m = 0.0;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) m = fmax(m, hypot(A[e].x, A[e].y));
  part[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] = fmax(part[threadIdx.x], part[threadIdx.x + w]);
    __syncthreads();
  }
  const double s = part[0];
  if (!(s > 0.0)) return;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) A[e] = make_double2(A[e].x / s, A[e].y / s);
}

// y += a x
__global__ void k_axpy(const double2* __restrict__ x, double2* y, long long n, double2 a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    y[e] = make_double2(y[e].x + a.x * v.x - a.y * v.y, y[e].y + a.x * v.y + a.y * v.x);
  }
}

unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152LL * 32) b = 152LL * 32;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_strided_copy(const double2* src, double2* dst, const StridedView& v, cudaStream_t s) {
  if (v.rank < 1 || v.rank > kStridedMaxRank || v.total <= 0) return v.total == 0 ? cudaSuccess : cudaErrorInvalidValue;
  k_strided_copy<<<blocks_for(v.total), 256, 0, s>>>(src, dst, v);
  return cudaGetLastError();
}

cudaError_t launch_pinv_rows(double2* W, const double2* Rem, int n, int ncols, double rcond, cudaStream_t s) {
  if (n <= 0 || ncols <= 0) return cudaSuccess;
  if ((size_t)n * sizeof(double) > 48 * 1024) return cudaErrorInvalidValue;
  k_pinv_rows<<<1, 256, (size_t)n * sizeof(double), s>>>(W, Rem, n, ncols, rcond);
  return cudaGetLastError();
}

cudaError_t launch_quad_form(const double2* T, const double2* X, long long n, double* out, cudaStream_t s) {
  k_quad_form<<<1, 256, 0, s>>>(T, X, n, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_absmax(double2* A, long long n, cudaStream_t s) {
  k_scale_absmax<<<1, 256, 0, s>>>(A, n);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double2* x, double2* y, long long n, double2 a, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_axpy<<<blocks_for(n), 256, 0, s>>>(x, y, n, a);
  return cudaGetLastError();
}

}  // namespace bbp
