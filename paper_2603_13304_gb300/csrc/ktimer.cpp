// Live timing of one kernel class with CUDA events on its launch stream.
//
// When a class is selected, every launch of it is bracketed by a pair of
// events recorded on the stream it is launched on (with the external-record
// flag when the stream is being captured, so that the pair becomes event
// nodes of the graph and every replay re-records it).  Pairs recorded eagerly are read
// once and dropped; pairs baked into a captured graph carry that graph's tag
// and are re-read after each replay until the graph is dropped.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace bbp {

namespace {

struct Pair {
  cudaEvent_t a = nullptr, b = nullptr;
  double flops = 0.0;
  long long tag = -1;
  long long gen = 0;   // selection during which the pair was recorded
};

std::mutex g_mu;
std::atomic<int> g_class{0};   // read on every launch path without the lock
std::vector<Pair> g_pairs;
long long g_n = 0;
long long g_gen = 0;
double g_ms = 0.0, g_flops = 0.0;
double* g_dev_flops = nullptr;   // kernels that count their own work add here
thread_local long long t_tag = -1;

void destroy(Pair& p) {
  if (p.a) cudaEventDestroy(p.a);
  if (p.b) cudaEventDestroy(p.b);
  p.a = p.b = nullptr;
}

}  // namespace

// A new selection drops the eager pairs only: pairs with a graph tag are
// event nodes of a captured graph that a live context may replay, so they
// stay valid until that graph is dropped (ktimer_drop_tag); they are no
// longer counted, because they belong to an earlier selection.
void ktimer_select(int cls) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<Pair> keep;
  for (Pair& p : g_pairs) {
    if (p.tag == -1) destroy(p);
    else keep.push_back(p);
  }
  g_pairs.swap(keep);
  ++g_gen;
  g_class = cls;
  g_n = 0;
  g_ms = g_flops = 0.0;
  if (cls && !g_dev_flops) {
    if (cudaMalloc(&g_dev_flops, sizeof(double)) != cudaSuccess) g_dev_flops = nullptr;
  }
  if (g_dev_flops) cudaMemset(g_dev_flops, 0, sizeof(double));
}

int ktimer_class() { return g_class.load(std::memory_order_relaxed); }

double* ktimer_device_flops(int cls) {
  const int c = g_class.load(std::memory_order_relaxed);
  return (c && c == cls) ? g_dev_flops : nullptr;
}

void ktimer_set_tag(long long tag) { t_tag = tag; }

void ktimer_drop_tag(long long tag) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<Pair> keep;
  for (Pair& p : g_pairs) {
    if (p.tag == tag) destroy(p);
    else keep.push_back(p);
  }
  g_pairs.swap(keep);
}

KTimerScope::KTimerScope(int cls, cudaStream_t s, double flops) : s_(s) {
  const int c = g_class.load(std::memory_order_relaxed);
  if (!c || cls != c) return;
  Pair p;
  if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
    destroy(p);
    return;
  }
  p.flops = flops;
  p.tag = t_tag;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    destroy(p);
    return;
  }
  external_ = cs == cudaStreamCaptureStatusActive;
  // a capture that the engine did not start (no graph tag): the caller's
  // graph would own the events, which eager collection destroys; not timed
  if (external_ && p.tag == -1) {
    destroy(p);
    return;
  }
  if ((external_ ? cudaEventRecordWithFlags(p.a, s, cudaEventRecordExternal) : cudaEventRecord(p.a, s)) != cudaSuccess) {
    cudaGetLastError();   // a failed timing record must not surface as the launch's error
    destroy(p);
    return;
  }
  a_ = p.a;
  b_ = p.b;
  std::lock_guard<std::mutex> lk(g_mu);
  p.gen = g_gen;
  g_pairs.push_back(p);
}

KTimerScope::~KTimerScope() {
  if (!b_) return;
  if ((external_ ? cudaEventRecordWithFlags(b_, s_, cudaEventRecordExternal) : cudaEventRecord(b_, s_)) != cudaSuccess)
    cudaGetLastError();
}

// Add the pairs of `tag` (all completed: the caller has synchronised) to the
// totals; eager pairs (tag -1) are dropped afterwards.
void ktimer_collect(long long tag) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_class) return;
  std::vector<Pair> keep;
  for (Pair& p : g_pairs) {
    if (p.tag != tag) {
      keep.push_back(p);
      continue;
    }
    float ms = 0.f;
    if (p.gen == g_gen && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms += ms;
      g_flops += p.flops;
      ++g_n;
    }
    if (tag == -1) destroy(p);
    else keep.push_back(p);
  }
  g_pairs.swap(keep);
}

void ktimer_read(long long* n, double* ms, double* flops) {
  std::lock_guard<std::mutex> lk(g_mu);
  double dev = 0.0;
  if (g_dev_flops) {
    cudaMemcpy(&dev, g_dev_flops, sizeof(double), cudaMemcpyDeviceToHost);
    cudaMemset(g_dev_flops, 0, sizeof(double));
  }
  *n = g_n;
  *ms = g_ms;
  *flops = g_flops + dev;
  g_n = 0;
  g_ms = g_flops = 0.0;
}

}  // namespace bbp
