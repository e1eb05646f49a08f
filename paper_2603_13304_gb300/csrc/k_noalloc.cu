// Allocation-free variant of the truncated-SVD entry point.
//
// Some callers cannot allocate device memory at the moment they need an SVD:
// real-time loops that must not enter the allocator (cudaMalloc can
// synchronise the device), or hosts whose device memory is owned by another
// runtime with a budget fixed at start-up.  For them
// this file keeps the SVD scratch in a fixed device array, so a call needs no
// allocation of its own.
//
// The array is created on a device when this module is loaded there.  With
// CUDA's lazy module loading (the default) that happens at the first call of
// the entry point on that device, which also looks up the array's device
// address (cudaGetSymbolAddress, once per device, with that device current;
// the array's name is only a host-side stand-in in host code).  That first
// call should therefore come before any stream capture starts.  The kernel
// timer (bbp_ktimer_select) does not time launches inside a capture that the
// library did not start, so a selected timer class records nothing there.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace bbp {

// Largest scratch this entry point can use: enough for a 512 x 512 matrix
// (svd_work_bytes(512, 512) = 8,394,752 bytes).  Every GPU that loads the
// library holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)8 * 1024 * 1024 + 64 * 1024;

static __device__ __align__(256) unsigned char g_svd_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

// Device address of the scratch array on the current device (looked up once
// per device).  Returns the CUDA error of the lookup, if any.
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_svd_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Same computation as launch_svd_trunc, with the scratch taken from the fixed
// array.  The SVD setup kernel rewrites every scratch word it later reads
// (working matrix, rotation accumulator, counters), so the previous call's
// contents never leak into this one.  Every call on a device shares that
// device's array: two calls that overlap on the same GPU (for example on two
// streams) race and corrupt each other's results.
cudaError_t launch_svd_trunc_noalloc(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, int* status,
                                     cudaStream_t s, bool* too_large) {
  *too_large = svd_work_bytes(m, n) > kNoAllocScratchBytes;
  if (*too_large) return cudaSuccess;
  void* work = nullptr;
  cudaError_t e = noalloc_scratch(&work);
  if (e != cudaSuccess) return e;
  return launch_svd_trunc(Z, m, n, chi, U, Rem, work, status, s);
}

}  // namespace bbp
