// BlockBP engine (see engine.h).  Every step of the message update runs in the
// CUDA kernels of k_core.cu; this file only sizes buffers, follows the sweep
// plans and enqueues launches.
#include "engine.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace bbp {

// ------------------------------------------------------------- allocation

namespace {
std::mutex g_alloc_mu;
void* (*g_alloc)(size_t, void*, void*) = nullptr;
void (*g_free)(void*, void*, void*) = nullptr;
void* g_user = nullptr;

template <typename C> C one_of();
template <> double2 one_of<double2>() { return make_double2(1.0, 0.0); }
template <> float2 one_of<float2>() { return make_float2(1.f, 0.f); }
template <typename C> C zero_of();
template <> double2 zero_of<double2>() { return make_double2(0.0, 0.0); }
template <> float2 zero_of<float2>() { return make_float2(0.f, 0.f); }

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// truncated SVD of one split, per element type (complex128: the randomised
// subspace iteration with b = 2 chi, exact Jacobi for small splits)
cudaError_t svd_call(const double2* Z, int m, int n, int chi, double2* U, double2* Rem, void* work, int* status,
                     cudaStream_t s, int power_iters, bool, int*) {
  return launch_svd_trunc_rand64(Z, m, n, chi, U, Rem, work, status, s, power_iters);
}

// Segment merge C (M x N) = A (M x K) B (K x N), row-major: on the tensor
// cores (split TF32, complex64 modes with tc) when the product is large
// enough to pay for packing, else the SIMT GEMM.
constexpr double kTcMergeMin = 1 << 22;   // complex multiply-adds
size_t merge_tc_bytes(int M, int N, int K) { return tc_zpack_bytes(false, M, K) + tc_zpack_bytes(false, 2 * N, K); }
cudaError_t merge_call(int M, int N, int K, const double2* A, const double2* B, double2* C, void*, size_t, int*,
                       bool, cudaStream_t s) {
  return launch_zgemm('N', 'N', M, N, K, make_double2(1, 0), A, K, 0, B, N, 0, make_double2(0, 0), C, N, 0, 1, s);
}
cudaError_t merge_call(int M, int N, int K, const float2* A, const float2* B, float2* C, void* tcw, size_t tcw_bytes,
                       int* tc_err, bool tc, cudaStream_t s) {
  if (tc && tcw && (double)M * N * K >= kTcMergeMin && merge_tc_bytes(M, N, K) <= tcw_bytes) {
    void* Bp = (char*)tcw + tc_zpack_bytes(false, M, K);
    cudaError_t e = tc_zpack_a(false, 'N', M, K, A, K, tcw, s);
    if (e == cudaSuccess) e = tc_zpack_b(false, 'N', K, N, B, N, Bp, s);
    if (e == cudaSuccess) e = tc_zgemm_packed(false, M, N, K, tcw, Bp, C, N, tc_err, s);
    return e;
  }
  return launch_zgemm('N', 'N', M, N, K, make_float2(1, 0), A, K, 0, B, N, 0, make_float2(0, 0), C, N, 0, 1, s);
}

// launches of one truncated SVD (statistics only)
long long svd_launches(int m, int n, int chi, bool c64, int q) {
  const int M = std::min(m, n);
  const int b = c64 ? rand_block(m, n, chi) : rand_block64(m, n, chi);
  if (b >= M) return 5;
  return 12 + 4 * q + (c64 ? 1 : 0);
}
cudaError_t svd_call(const float2* Z, int m, int n, int chi, float2* U, float2* Rem, void* work, int* status,
                     cudaStream_t s, int power_iters, bool tensor_cores, int* tc_err) {
  return launch_svd_trunc(Z, m, n, chi, U, Rem, work, status, s, power_iters, tensor_cores, tc_err);
}
}  // namespace

void set_allocator(void* (*a)(size_t, void*, void*), void (*f)(void*, void*, void*), void* user) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = a;
  g_free = f;
  g_user = user;
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc(bytes, (void*)s, g_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (g_free) { g_free(p, (void*)s, g_user); return; }
  cudaFree(p);
}

bool DBuf::ensure(size_t n, cudaStream_t st) {
  if (n <= bytes && p) return true;
  release();
  p = dev_alloc(n, st);
  if (!p) { bytes = 0; return false; }
  bytes = n;
  s = st;
  return true;
}

void DBuf::release() {
  if (p) dev_free(p, s);
  p = nullptr;
  bytes = 0;
}

// Makes `dev` current for the scope and restores the caller's device after.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (dev < 0 || cudaGetDevice(&prev) != cudaSuccess || prev == dev) { prev = -1; return; }
    if (cudaSetDevice(dev) != cudaSuccess) prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int fail(Engine* e, int status, const std::string& msg) {
  if (e) e->last_error = msg;
  return status;
}

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t _e = (call);                                                                          \
    if (_e != cudaSuccess) return fail(this, 3, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// ------------------------------------------------------------ sweep work

bool SweepWork::reserve(size_t el, size_t ct, size_t cs, size_t cx, size_t sb, size_t ns, size_t cd, size_t tb) {
  if (el == elem && ct <= cap_t && cs <= cap_seg && cx <= cap_x && sb <= svd_bytes && ns <= nslots && cd <= cap_d &&
      tb <= tc_bytes && arena.p)
    return true;
  if (el != elem) { cap_t = cap_seg = cap_x = svd_bytes = nslots = cap_d = tc_bytes = 0; }
  ++gen;                               // the layout changes (even when the base address comes back)
  tc_bytes = std::max(tb, tc_bytes);
  elem = el;
  cap_t = std::max(ct, cap_t);
  cap_seg = std::max(cs, cap_seg);
  cap_x = std::max(cx, cap_x);
  svd_bytes = std::max(sb, svd_bytes);
  nslots = std::max(ns, nslots);
  cap_d = std::max(cd, cap_d);
  const size_t z = elem, zd = sizeof(double2);
  size_t total = nslots * al(cap_t * z) + 4 * al(cap_seg * z) + 3 * al(cap_t * z) + al(4096 * z) + al(cap_x * z) +
                 al(svd_bytes) + 256 * 4 + al(64 * sizeof(void*) * 2) + al(64 * 3 * 2 * sizeof(int)) +
                 al((2 * 64 * 64 + 64 * 64 * 64 + 256) * zd) + 4 * al(cap_d * zd) + al(4096 * zd) + al(tc_bytes);
  if (!arena.ensure(total, stream)) return false;
  char* p = (char*)arena.p;
  slot.assign(nslots, nullptr);
  for (size_t i = 0; i < nslots; ++i) { slot[i] = p; p += al(cap_t * z); }
  for (int i = 0; i < 2; ++i) { S[i] = p; p += al(cap_seg * z); }
  for (int i = 0; i < 2; ++i) { R[i] = p; p += al(cap_seg * z); }
  qrA = p; p += al(cap_t * z);
  qrQ = p; p += al(cap_t * z);
  qrR = p; p += al(cap_t * z);
  tau = p; p += al(4096 * z);
  X = p; p += al(cap_x * z);
  svd = p; p += al(svd_bytes);
  logscale = (double*)p; p += 256;
  status = (int*)p; p += 256;
  scal = (double2*)p; p += 256;
  p += 256;
  ptrs = (void**)p; p += al(64 * sizeof(void*) * 2);
  ints = (int*)p; p += al(64 * 3 * 2 * sizeof(int));
  k4 = (double2*)p; p += al((2 * 64 * 64 + 64 * 64 * 64 + 256) * zd);
  dX0 = (double2*)p; p += al(cap_d * zd);
  dX1 = (double2*)p; p += al(cap_d * zd);
  dQ = (double2*)p; p += al(cap_d * zd);
  dR = (double2*)p; p += al(cap_d * zd);
  dtau = (double2*)p; p += al(4096 * zd);
  tc = tc_bytes ? (void*)p : nullptr;
  p += al(tc_bytes);
  return true;
}

// ---------------------------------------------------------------- engine

void Engine::drop_graphs() {
  for (int p = 0; p < 2; ++p) {
    if (graphs[p].exec) cudaGraphExecDestroy(graphs[p].exec);
    if (graphs[p].graph) cudaGraphDestroy(graphs[p].graph);
    graphs[p] = IterGraph();
    ktimer_drop_tag(graph_tag(p));
  }
}

namespace {
std::atomic<unsigned long long> g_uid{1};
}

bool Engine::deferred(Deferred& d) const {
  if (!in_flight || !pending_launch) return false;
  const IterGraph& g = graphs[launched_parity];
  const int nu = (int)geom.updates().size();
  double* tol_dev = (double*)((char*)dist_dev.p + ((sizeof(double) * nu + 2 * sizeof(int) * nu + 255) & ~size_t(255)));
  d.graph = g.graph;
  d.uid = g.uid;
  d.tol_dev = tol_dev;
  d.word_dev = tol_dev + 4;
  d.host_word = h_word;
  d.pool = workers.get();
  return g.graph != nullptr;
}

int Engine::defer_before(cudaStream_t batch) {
  DeviceScope ds(device);
  if (!root_pre) CK(cudaEventCreateWithFlags(&root_pre, cudaEventDisableTiming));
  CK(cudaEventRecord(root_pre, root));
  CK(cudaStreamWaitEvent(batch, root_pre, 0));
  if (workers) CK(cudaStreamWaitEvent(batch, workers->last_done, 0));
  return 0;
}

int Engine::defer_after(cudaStream_t batch) {
  DeviceScope ds(device);
  CK(cudaEventRecord(root_out, batch));
  CK(cudaStreamWaitEvent(root, root_out, 0));
  if (workers) {
    std::lock_guard<std::mutex> lk(workers->mu);
    CK(cudaEventRecord(workers->last_done, batch));
    auto& pv = workers->pending;
    pv.erase(std::remove(pv.begin(), pv.end(), this), pv.end());
  }
  pending_launch = false;
  return 0;
}

int Engine::launch_deferred_now() {
  DeviceScope ds(device);
  if (!pending_launch) return 0;
  IterGraph& g = graphs[launched_parity];
  const int nu = (int)geom.updates().size();
  double* tol_dev = (double*)((char*)dist_dev.p + ((sizeof(double) * nu + 2 * sizeof(int) * nu + 255) & ~size_t(255)));
  double* word_dev = tol_dev + 4;
  if (!g.exec) {
    const cudaError_t ce = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (ce != cudaSuccess) return fail(this, 3, std::string("graph instantiation: ") + cudaGetErrorString(ce));
  }
  CK(cudaStreamWaitEvent(root, workers->last_done, 0));
  CK(cudaMemcpyAsync(tol_dev, h_word, sizeof(double), cudaMemcpyHostToDevice, root));
  CK(cudaGraphLaunch(g.exec, root));
  CK(cudaMemcpyAsync(h_word + 1, word_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, root));
  CK(cudaEventRecord(root_out, root));
  CK(cudaEventRecord(workers->last_done, root));
  pending_launch = false;
  return 0;
}

// FNV-1a over everything a captured iteration bakes in: job tensors and
// shapes, destination buffers and the workspace arenas.
unsigned long long Engine::iter_signature(const std::vector<SweepJob>& jobs, int nstreams) const {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  auto mixs = [&](const TShape& t) { mix((unsigned long long)t.l); mix((unsigned long long)t.p); mix((unsigned long long)t.r); };
  mix((unsigned long long)precision);
  mix(tc_tune_generation());           // the tensor-core tiles the launches take
  mix((unsigned long long)chi);
  mix((unsigned long long)power_iters);
  mix((unsigned long long)power_iters64);
  {
    unsigned long long ab;
    std::memcpy(&ab, &alpha, sizeof ab);
    mix(ab);
  }
  mix((unsigned long long)hermitise);
  mix((unsigned long long)nstreams);
  mix((unsigned long long)(uintptr_t)dist_dev.p);
  for (int i = 0; i < nstreams; ++i) {
    mix((unsigned long long)(uintptr_t)workers->w[i]->arena.p);
    mix(workers->w[i]->gen);
  }
  for (const SweepJob& j : jobs) {
    mix((unsigned long long)(uintptr_t)j.plan);
    for (const void* p : j.node_tensor) mix((unsigned long long)(uintptr_t)p);
    for (const auto& f : j.node_fuse) mix((unsigned long long)(f[0] + 1) * 256 + f[1] * 64 + f[2] * 16 + f[3] * 4 + f[4]);
    for (const TShape& t : j.node_shape) mixs(t);
    for (const void* p : j.start) mix((unsigned long long)(uintptr_t)p);
    for (const TShape& t : j.start_shape) mixs(t);
    for (const void* p : j.dest) mix((unsigned long long)(uintptr_t)p);
    for (const TShape& t : j.tr.final_mps) mixs(t);
  }
  return h;
}

// What a captured iteration reads, without simulating it: every message's
// current shapes and buffers, the fused tensors' buffers and the workspaces.
// Equal input signatures imply equal job signatures (the plans are fixed).
unsigned long long Engine::input_signature(int nstreams) const {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  mix((unsigned long long)precision);
  mix((unsigned long long)tc_mode);
  mix(tc_tune_generation());
  mix((unsigned long long)chi);
  mix((unsigned long long)power_iters);
  mix((unsigned long long)power_iters64);
  {
    unsigned long long ab;
    std::memcpy(&ab, &alpha, sizeof ab);
    mix(ab);
  }
  mix((unsigned long long)hermitise);
  mix((unsigned long long)nstreams);
  mix((unsigned long long)(uintptr_t)dist_dev.p);
  for (int i = 0; workers && i < nstreams && i < (int)workers->w.size(); ++i) {
    mix((unsigned long long)(uintptr_t)workers->w[i]->arena.p);
    mix(workers->w[i]->gen);
  }
  for (const auto& kv : msgs) {
    const Message& m = kv.second;
    mix((unsigned long long)m.cur);
    mix((unsigned long long)(uintptr_t)m.buf[0].p);
    mix((unsigned long long)(uintptr_t)m.buf[1].p);
    for (const TShape& t : m.sh[m.cur]) {
      mix((unsigned long long)t.l);
      mix((unsigned long long)t.p);
      mix((unsigned long long)t.r);
    }
  }
  for (const auto& kv : fused) mix((unsigned long long)(uintptr_t)kv.second.p);
  return h;
}

Engine::~Engine() {
  if (workers) {
    std::lock_guard<std::mutex> lk(workers->mu);
    auto& pv = workers->pending;
    pv.erase(std::remove(pv.begin(), pv.end(), this), pv.end());
  }
  drop_graphs();
  if (root) {
    cudaStreamSynchronize(root);
    cudaStreamDestroy(root);
  }
  if (root_in) cudaEventDestroy(root_in);
  if (root_in2) cudaEventDestroy(root_in2);
  if (root_out) cudaEventDestroy(root_out);
  if (root_pre) cudaEventDestroy(root_pre);
  if (h_word) cudaFreeHost(h_word);
  workers.reset();
}

WorkerPool::WorkerPool() { cudaEventCreateWithFlags(&last_done, cudaEventDisableTiming); }

WorkerPool::~WorkerPool() {
  if (last_done) {
    cudaEventSynchronize(last_done);
    cudaEventDestroy(last_done);
  }
  for (SweepWork* x : w) {
    if (x->stream) cudaStreamSynchronize(x->stream);
    x->arena.release();
    if (x->done) cudaEventDestroy(x->done);
    if (x->stream) cudaStreamDestroy(x->stream);
    delete x;
  }
}

WorkerPool& Engine::pool_ref() {
  if (!workers) workers = std::make_shared<WorkerPool>();
  return *workers;
}

int Engine::use_workers(std::shared_ptr<WorkerPool> p) {
  DeviceScope ds(device);
  if (root) CK(cudaStreamSynchronize(root));
  if (stream) CK(cudaStreamSynchronize(stream));
  if (workers) CK(cudaEventSynchronize(workers->last_done));
  drop_graphs();
  workers = p ? std::move(p) : std::make_shared<WorkerPool>();
  return 0;
}

SweepWork* Engine::work(size_t i) {
  WorkerPool& P = pool_ref();
  while (P.w.size() <= i) {
    SweepWork* w = new SweepWork();
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) { delete w; return nullptr; }
    cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming);
    P.w.push_back(w);
  }
  return P.w[i];
}

int Engine::create(int lattice, int Lx, int Ly, int periodic, int d_, int D_, const double* host_t, cudaStream_t s) {
  if (d_ < 1 || d_ > 4 || D_ < 1 || D_ > 8) return fail(this, 1, "d must be 1..4 and D 1..8");
  if (!host_t) return fail(this, 1, "host_tensors is NULL");
  if (lattice != 0 && lattice != 1) return fail(this, 1, "lattice must be BBP_SQUARE or BBP_KAGOME");
  if (Lx <= 0 || Ly <= 0 || Lx > 4096 || Ly > 4096) return fail(this, 1, "lattice size out of range");
  if (lattice == 1 && !periodic) return fail(this, 1, "Kagome lattices are periodic super-cells");
  d = d_;
  D = D_;
  stream = s;
  uid_ = g_uid.fetch_add(1);
  if (cudaGetDevice(&device) != cudaSuccess) return fail(this, 3, "no current CUDA device");
  geom.lat.kind = lattice;
  geom.lat.Lx = Lx;
  geom.lat.Ly = Ly;
  geom.lat.periodic = periodic != 0;
  const int n = geom.lat.n_sites();
  const size_t per = (size_t)d * D * D * D * D;
  {
    cudaError_t ae = init_kernel_attributes();
    if (ae != cudaSuccess) return fail(this, 3, std::string("kernel attributes: ") + cudaGetErrorString(ae));
  }
  if (!t_dev.ensure(sizeof(double2) * per * n, s)) return fail(this, 2, "device allocation of site tensors failed");
  CK(cudaMemcpyAsync(t_dev.p, host_t, sizeof(double2) * per * n, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return 0;
}

int Engine::partition(int bx, int by) {
  std::string err = geom.build(geom.lat.kind, geom.lat.Lx, geom.lat.Ly, geom.lat.periodic, bx, by);
  if (!err.empty()) return fail(this, 4, err);
  const int n = geom.lat.n_sites();
  site_n.assign(n, {D, D, D, D});
  for (const Block& b : geom.blocks)
    for (size_t q = 0; q < b.sites.size(); ++q) {
      int t = b.sites[q][0], i = b.sites[q][1], j = b.sites[q][2];
      for (int k = 0; k < 4; ++k) {
        int t2, i2, j2, k2;
        geom.lat.neighbour(t, i, j, k, t2, i2, j2, k2);
        if (geom.lat.site_id(t2, i2, j2) < 0) site_n[b.gids[q]][k] = 1;
      }
    }
  block_regions.assign(geom.blocks.size(), Region());
  for (const Block& b : geom.blocks) {
    err = build_region(geom, {{b.X, b.Y}}, block_regions[b.id]);
    if (!err.empty()) return fail(this, 4, err);
  }
  plans.clear();
  for (const auto& u : geom.updates()) {
    SweepPlan plan;
    err = compile_sweep(geom, block_regions[u.block], u.face, plan);
    if (!err.empty()) return fail(this, 4, "sweep plan: " + err);
    plans[{u.block, u.face}] = std::move(plan);
  }
  msgs.clear();
  for (const Block& b : geom.blocks)
    for (int f = 0; f < 4; ++f) {
      Message& m = msgs[{b.id, f}];
      m.open = b.faces[f].nbr < 0;
      for (const Edge& e : b.faces[f].edges) m.Dleg.push_back(e.gid < 0 ? 1 : D);
    }
  fused.clear();
  partitioned = true;
  messages_ready = false;
  return 0;
}

int Engine::set_precision(int p) {
  if (p < 0 || p > 2) return fail(this, 1, "unknown precision");
  if (messages_ready) return fail(this, 8, "precision must be set before bbp_init_messages");
  if (p != precision) fused.clear();
  precision = p;
  return 0;
}

// Whether the fused double-layer tensors of every site and sweep direction
// (at most four orders a site) would take more than fuse_cache_max; then
// each is fused (K1) into the sweep's scratch right before its absorb.
bool Engine::fuse_on_the_fly() const {
  size_t tot = 0;
  for (const auto& nn : site_n) {
    size_t e = 1;
    for (int q = 0; q < 4; ++q) e *= (size_t)nn[q] * nn[q];
    tot += 4 * e * elem();
  }
  return tot > fuse_cache_max;
}

template <typename C>
const C* Engine::fused_tensor(int gid, const int perm[4]) {
  int code = ((perm[0] * 4 + perm[1]) * 4 + perm[2]) * 4 + perm[3];
  auto key = std::make_pair(gid, code);
  auto it = fused.find(key);
  if (it != fused.end()) return (const C*)it->second.p;
  const auto& nn = site_n[gid];
  size_t tot = 1;
  for (int q = 0; q < 4; ++q) tot *= (size_t)nn[q] * nn[q];
  DBuf& b = fused[key];
  if (!b.ensure(tot * sizeof(C), stream)) { fused.erase(key); return nullptr; }
  const double2* t = (const double2*)t_dev.p + (size_t)gid * d * D * D * D * D;
  if (launch_fuse(t, d, D, nn.data(), nullptr, perm, (C*)b.p, stream) != cudaSuccess) return nullptr;
  return (const C*)b.p;
}

int Engine::init_messages(const double* edge_mats) {
  return precision == 0 ? init_messages_t<double2>(edge_mats) : init_messages_t<float2>(edge_mats);
}

template <typename C>
int Engine::init_messages_t(const double* edge_mats) {
  if (!partitioned) return fail(this, 8, "bbp_partition_blocks must come first");
  if (!edge_mats) return fail(this, 1, "edge_mats is NULL");
  const size_t cap = (size_t)chi * chi * D * D;
  std::vector<C> host;
  SweepWork* w = work(0);
  if (!w) return fail(this, 3, "stream creation failed");
  if (!w->reserve(sizeof(C), 16, 16, 16, 4096, 4, 16, 0)) return fail(this, 2, "work allocation failed");
  for (auto& kv : msgs) {
    Message& m = kv.second;
    const Block& b = geom.blocks[kv.first.first];
    const Face& f = b.faces[kv.first.second];
    if (m.open) {
      m.cap = 1;
      for (int which = 0; which < 2; ++which) {
        if (!m.buf[which].ensure(sizeof(C) * m.k(), stream)) return fail(this, 2, "message allocation failed");
        CK(launch_fill((C*)m.buf[which].p, m.k(), 1.0, 0.0, stream));
        m.sh[which].assign(m.k(), TShape{1, 1, 1});
      }
      m.cur = 0;
      continue;
    }
    m.cap = cap;
    for (int which = 0; which < 2; ++which)
      if (!m.buf[which].ensure(sizeof(C) * cap * m.k(), stream)) return fail(this, 2, "message allocation failed");
    host.assign(cap * m.k(), zero_of<C>());
    m.sh[0].clear();
    for (int q = 0; q < m.k(); ++q) {
      const Edge& e = f.edges[q];
      int g = b.gids[e.site];
      const double* src = edge_mats + ((size_t)g * 4 + e.slot) * D * D * 2;
      for (int a = 0; a < D * D; ++a) {
        C v;
        v.x = (decltype(v.x))src[2 * a];
        v.y = (decltype(v.y))src[2 * a + 1];
        host[(size_t)q * cap + a] = v;
      }
      m.sh[0].push_back(TShape{1, D * D, 1});
    }
    m.cur = 0;
    m.sh[1] = m.sh[0];
    CK(cudaMemcpyAsync(m.buf[0].p, host.data(), sizeof(C) * host.size(), cudaMemcpyHostToDevice, stream));
    int rc = finalize_message<C>(m, 0, *w, stream, nullptr, false);
    if (rc) return rc;
    CK(cudaStreamSynchronize(stream));
  }
  messages_ready = true;
  return 0;
}

// Normalise (unit norm, <I|M> > 0) buffer `which` of m on stream s;
// optionally write ||new - old|| (complex128 QR sweep) into dist_slot.
namespace {
template <typename C>
ChainDesc chain_of(const Message& m, int which) {
  ChainDesc d{};
  d.k = m.k();
  for (int q = 0; q < d.k; ++q) {
    d.T[q] = m.tensor<C>(which, q);
    d.l[q] = m.sh[which][q].l;
    d.p[q] = m.sh[which][q].p;
    d.r[q] = m.sh[which][q].r;
    d.D[q] = m.Dleg[q];
  }
  return d;
}
}  // namespace

// ------------------------------------------ learning step, Hermitisation
//
// Sec. 2.3.3: the message that replaces the old one is alpha new +
// (1 - alpha) old (Eq. of the learning step), and a message may be replaced
// by its Hermitian part (M + M^dagger) / 2 ("Hermitize MPSs").  Both are MPS
// sums: the direct sum of the two MPSs, compressed back to bond chi by a
// left-canonical QR sweep and a right-to-left truncated-SVD sweep, then
// normalised like every message.  The new message is Hermitised first.
// The shapes are fixed by the input shapes, so the host knows them at
// enqueue time (and a captured iteration replays them).

int Engine::reserve_learning(Message& m) {
  if (!learning() || m.open) return 0;
  const size_t bytes = elem() * (size_t)m.k() * 5 * m.cap;
  if (m.lrn.bytes >= bytes && m.lrn.p) return 0;
  CK(cudaStreamSynchronize(stream));
  if (!m.lrn.ensure(bytes, stream)) return fail(this, 2, "learning-step scratch allocation failed");
  return 0;
}

// compress the sum tensors held in m.lrn (shapes sh) to bond chi, in place
template <typename C>
int Engine::compress_lrn(Message& m, std::vector<TShape>& sh, SweepWork& w, cudaStream_t s) {
  const int k = (int)sh.size();
  const size_t cap4 = 4 * m.cap;
  C* aux = (C*)m.lrn.p;
  auto T = [&](int q) { return aux + (size_t)q * cap4; };
  const C one = one_of<C>(), zero = zero_of<C>();
  C* qrA = (C*)w.qrA;
  C* qrQ = (C*)w.qrQ;
  C* qrR = (C*)w.qrR;
  C* tau = (C*)w.tau;
  C* S0 = (C*)w.S[0];
  for (int q = 0; q + 1 < k; ++q) {   // left-canonical QR sweep
    const TShape a = sh[q], b = sh[q + 1];
    const int mm = a.l * a.p, nn = a.r, kk = std::min(mm, nn);
    CK(cudaMemcpyAsync(qrA, T(q), sizeof(C) * (size_t)mm * nn, cudaMemcpyDeviceToDevice, s));
    CK(launch_qr(qrA, mm, nn, qrQ, qrR, tau, s));
    CK(cudaMemcpyAsync(T(q), qrQ, sizeof(C) * (size_t)mm * kk, cudaMemcpyDeviceToDevice, s));
    sh[q].r = kk;
    CK(launch_zgemm('N', 'N', kk, b.p * b.r, nn, one, qrR, nn, 0, T(q + 1), b.p * b.r, 0, zero, S0, b.p * b.r, 0, 1,
                    s));
    CK(cudaMemcpyAsync(T(q + 1), S0, sizeof(C) * (size_t)kk * b.p * b.r, cudaMemcpyDeviceToDevice, s));
    sh[q + 1].l = kk;
    sweep_launches += 5;
  }
  for (int q = k - 1; q >= 1; --q) {  // truncated SVDs from the right: Z^H = U' Rem', T_q = U'^H
    const TShape a = sh[q], b = sh[q - 1];
    const int l = a.l, pr = a.p * a.r, kk = std::min(chi, std::min(pr, l));
    CK(launch_conj_transpose(T(q), l, pr, qrA, s));
    const bool c64 = sizeof(C) == sizeof(float2);
    const int qsteps = c64 ? power_iters : power_iters64;
    CK(svd_call(qrA, pr, l, chi, qrQ, qrR, w.svd, w.status, s, qsteps, false, w.status + 1));
    CK(launch_conj_transpose(qrQ, pr, kk, T(q), s));
    sh[q].l = kk;
    CK(launch_zgemm('N', 'C', b.l * b.p, kk, l, one, T(q - 1), l, 0, qrR, l, 0, zero, S0, kk, 0, 1, s));
    CK(cudaMemcpyAsync(T(q - 1), S0, sizeof(C) * (size_t)b.l * b.p * kk, cudaMemcpyDeviceToDevice, s));
    sh[q - 1].r = kk;
    sweep_launches += 4 + svd_launches(pr, l, chi, c64, qsteps);
  }
  return 0;
}

// Hermitisation and the learning step of the new message in buffer `which`
// (shapes m.sh[which], updated); the old message is buffer 1 - which.
template <typename C>
int Engine::learn_message(Message& m, int which, SweepWork& w, cudaStream_t s) {
  const int k = m.k();
  const size_t cap4 = 4 * m.cap;
  C* aux = (C*)m.lrn.p;
  C* dag = aux + (size_t)k * cap4;
  auto T = [&](int q) { return aux + (size_t)q * cap4; };
  auto sum_into = [&](C* const* x, const std::vector<TShape>& xs, C* const* y, const std::vector<TShape>& ys,
                      double2 ca, double2 cb, std::vector<TShape>& out) -> int {
    out.assign(k, TShape());
    for (int q = 0; q < k; ++q) {
      CK(launch_mps_sum(x[q], xs[q].l, xs[q].r, y[q], ys[q].l, ys[q].r, xs[q].p, q, k, ca, cb, T(q), s));
      out[q].l = (k == 1 || q == 0) ? xs[q].l : xs[q].l + ys[q].l;
      out[q].p = xs[q].p;
      out[q].r = (k == 1 || q == k - 1) ? xs[q].r : xs[q].r + ys[q].r;
    }
    sweep_launches += k;
    return 0;
  };
  auto store_back = [&](const std::vector<TShape>& sh) -> int {
    for (int q = 0; q < k; ++q) {
      if ((size_t)sh[q].size() > m.cap) return fail(this, 8, "learned message tensor exceeds its buffer");
      CK(cudaMemcpyAsync(m.tensor<C>(which, q), T(q), sizeof(C) * (size_t)sh[q].size(), cudaMemcpyDeviceToDevice, s));
    }
    m.sh[which] = sh;
    CK(launch_msg_normalise(chain_of<C>(m, which), sizeof(C) == sizeof(float2), w.k4, s));
    sweep_launches += k + 1;
    return 0;
  };
  std::vector<C*> nw(k), od(k), dg(k);
  for (int q = 0; q < k; ++q) {
    nw[q] = m.tensor<C>(which, q);
    od[q] = m.tensor<C>(1 - which, q);
    dg[q] = dag + (size_t)q * m.cap;
  }
  std::vector<TShape> sh;
  if (hermitise) {
    for (int q = 0; q < k; ++q) {
      const TShape t = m.sh[which][q];
      CK(launch_mps_dagger(nw[q], t.l, m.Dleg[q], t.r, dg[q], s));
    }
    if (int rc = sum_into(nw.data(), m.sh[which], dg.data(), m.sh[which], make_double2(0.5, 0), make_double2(0.5, 0), sh))
      return rc;
    if (int rc = compress_lrn<C>(m, sh, w, s)) return rc;
    if (int rc = store_back(sh)) return rc;
  }
  if (alpha != 1.0) {
    if (int rc = sum_into(nw.data(), m.sh[which], od.data(), m.sh[1 - which], make_double2(alpha, 0),
                          make_double2(1.0 - alpha, 0), sh))
      return rc;
    if (int rc = compress_lrn<C>(m, sh, w, s)) return rc;
    if (int rc = store_back(sh)) return rc;
  }
  return 0;
}

// Normalise (unit norm, <I|M> > 0) buffer `which` of m on stream s;
// optionally write ||new - old|| into dist_slot: the norm of the direct-sum
// MPS (new, -old) reduced by a QR sweep, in the element type (absolute
// accuracy ~ eps of that type, no sqrt(2 - 2 Re<old|new>) floor).  In an
// iteration (with_distance) the learning step and the Hermitisation come
// between the two.
template <typename C>
int Engine::finalize_message(Message& m, int which, SweepWork& w, cudaStream_t s, double* dist_slot,
                             bool with_distance) {
  const int k = m.k();
  if (k > kMaxChain) return fail(this, 1, "message longer than 64 tensors");
  CK(launch_msg_normalise(chain_of<C>(m, which), sizeof(C) == sizeof(float2), w.k4, s));
  sweep_launches += 1;
  if (!with_distance) return 0;
  if (learning() && !m.open)
    if (int rc = learn_message<C>(m, which, w, s)) return rc;
  const int old = 1 - which;
  const C one = one_of<C>(), zero = zero_of<C>();
  C* X0 = (C*)w.dX0;
  C* X1 = (C*)w.dX1;
  C* Qd = (C*)w.dQ;
  C* Rd = (C*)w.dR;
  int kprev = 0;
  for (int q = 0; q < k; ++q) {
    const TShape& a = m.sh[which][q];
    const TShape& b = m.sh[old][q];
    const int L = (k == 1 || q == 0) ? 1 : a.l + b.l;
    const int Rr = (k == 1 || q == k - 1) ? 1 : a.r + b.r;
    const int p = a.p;
    CK(launch_direct_sum(m.tensor<C>(which, q), a.l, a.r, m.tensor<C>(old, q), b.l, b.r, p, q, k, X0, s));
    C* X = X0;
    int rows = L;
    if (q > 0) {
      CK(launch_zgemm('N', 'N', kprev, p * Rr, L, one, Rd, L, 0, X0, p * Rr, 0, zero, X1, p * Rr, 0, 1, s));
      X = X1;
      rows = kprev;
    }
    const int mrows = rows * p;
    CK(launch_qr_r(X, mrows, Rr, Rd, Qd, X == X1 ? X0 : X1, s));
    kprev = std::min(mrows, Rr);
    sweep_launches += 3;
  }
  CK(launch_frob(Rd, (long long)kprev, dist_slot, s));
  sweep_launches += 1;
  return 0;
}

template <typename C>
int Engine::fill_job(const Region& R, const SweepPlan& plan, SweepJob& job, const OpList& ops,
                     std::vector<DBuf*>& tmp) {
  job.plan = &plan;
  LegDims dims;
  job.node_tensor.assign(plan.nodes.size(), nullptr);
  job.node_fuse.assign(plan.nodes.size(), std::array<int, 5>{-1, 0, 0, 0, 0});
  job.node_shape.assign(plan.nodes.size(), TShape());
  dims.node_dims.resize(plan.nodes.size());
  for (size_t s = 0; s < plan.nodes.size(); ++s) {
    const SweepNode& n = plan.nodes[s];
    const SweepStep& st = plan.steps[s];
    if (n.site) {
      const auto& nn = site_n[n.gid];
      for (int k = 0; k < 4; ++k) dims.node_dims[s][k] = nn[k] * nn[k];
      int perm[4];
      for (int q = 0; q < st.nin; ++q) perm[q] = st.in_leg[q];
      for (int q = 0; q < st.nout; ++q) perm[st.nin + q] = st.out_leg[q];
      const double* op = nullptr;
      for (const auto& o : ops)
        if (o.first[0] == n.inst && o.first[1] == n.local) op = o.second;
      if (op) {
        size_t tot = 1;
        for (int q = 0; q < 4; ++q) tot *= (size_t)nn[q] * nn[q];
        DBuf* b = new DBuf();
        tmp.push_back(b);
        if (!b->ensure(tot * sizeof(C), stream)) return fail(this, 2, "fused operator allocation failed");
        const double2* t = (const double2*)t_dev.p + (size_t)n.gid * d * D * D * D * D;
        CK(launch_fuse(t, d, D, nn.data(), (const double2*)op, perm, (C*)b->p, stream));
        job.node_tensor[s] = b->p;
      } else if (fuse_on_the_fly()) {
        job.node_tensor[s] = nullptr;  // fused into the sweep's scratch right before its absorb
        job.node_fuse[s] = {n.gid, perm[0], perm[1], perm[2], perm[3]};
      } else {
        job.node_tensor[s] = fused_tensor<C>(n.gid, perm);
        if (!job.node_tensor[s]) return fail(this, 2, "fusion failed");
      }
    } else {
      const Message& m = msgs.at({R.ids[n.msg_inst], n.msg_dir});
      const TShape sh = m.sh[m.cur][n.msg_index];
      job.node_shape[s] = sh;
      job.node_tensor[s] = m.tensor<C>(m.cur, n.msg_index);
      dims.node_dims[s] = {sh.l, sh.p, sh.r, 1};
    }
  }
  job.start.clear();
  job.start_shape.clear();
  for (const auto& st : plan.start) {
    const Message& m = msgs.at({R.ids[st[0]], st[1]});
    job.start.push_back(m.tensor<C>(m.cur, st[2]));
    job.start_shape.push_back(m.sh[m.cur][st[2]]);
    dims.start.push_back(m.sh[m.cur][st[2]]);
  }
  std::string err = simulate_shapes(plan, dims, chi, job.tr);
  if (!err.empty()) return fail(this, 8, "shape simulation: " + err);
  return 0;
}

// Workspace (in elements, except the SVD bytes) needed by one sweep job.
void Engine::job_needs(const SweepJob& job, size_t need[7]) const {
  const ShapeTrace& tr = job.tr;
  size_t cap_x = 1;
  for (size_t q = 0; q < job.plan->nodes.size(); ++q) {
    if (!job.plan->nodes[q].site) cap_x = std::max(cap_x, (size_t)job.node_shape[q].size());
    else if (job.node_fuse[q][0] >= 0) {
      const auto& nn = site_n[job.node_fuse[q][0]];
      size_t tot = 1;
      for (int k = 0; k < 4; ++k) tot *= (size_t)nn[k] * nn[k];
      cap_x = std::max(cap_x, tot);
    }
  }
  const int mr = (int)std::max<long long>(tr.max_svd_rows, 1), mc = (int)std::max<long long>(tr.max_svd_cols, 1);
  need[0] = std::max<size_t>(need[0], (size_t)tr.max_tensor);
  need[1] = std::max<size_t>(need[1], (size_t)std::max(tr.max_seg, tr.max_tensor));
  need[2] = std::max<size_t>(need[2], cap_x);
  need[3] = std::max<size_t>(need[3], precision == 0 ? svd_work_bound_rand64(mr, mc, chi)
                                                     : svd_work_bound_c64(mr, mc, chi, false));
  need[4] = std::max<size_t>(need[4], (size_t)tr.max_len + 6);
  need[5] = std::max<size_t>(need[5], (size_t)4 * chi * chi * D * D + 64);
  if (tc_mode && precision != 0)
    for (const auto& st : tr.steps)
      need[6] = std::max<size_t>(need[6], tc_absorb_bytes(tc_mode == 2, st.P, st.Q, st.l, st.r));
  if (learning()) {
    // compression of a direct sum: tensors up to (2 chi) x D^2 x (2 chi); SVDs of (2 chi D^2) x (2 chi)
    const size_t s4 = (size_t)4 * chi * chi * D * D;
    need[0] = std::max(need[0], s4);
    need[1] = std::max(need[1], s4);
    const int lr = 2 * chi * D * D, lc = 2 * chi;
    need[3] = std::max<size_t>(need[3], precision == 0 ? svd_work_bound_rand64(lc, lr, chi)
                                                       : svd_work_bound_c64(lc, lr, chi, false));
  }
}

int Engine::reserve_workers(const std::vector<SweepJob>& jobs, int nstreams) {
  for (int i = 0; i < nstreams; ++i) {
    size_t need[7] = {1, 1, 1, 256, 4, 16, 0};
    for (size_t j = i; j < jobs.size(); j += nstreams) job_needs(jobs[j], need);
    SweepWork& w = *workers->w[i];
    if (w.elem == elem() && need[0] <= w.cap_t && need[1] <= w.cap_seg && need[2] <= w.cap_x &&
        need[3] <= w.svd_bytes && need[4] <= w.nslots && need[5] <= w.cap_d && need[6] <= w.tc_bytes && w.arena.p)
      continue;
    // the arenas move: iterations of the pool's other members that are
    // bound to them and still wait for a batch launch run now, and every
    // use of the old arenas completes first
    for (Engine* e : workers->pending)
      if (e != this)
        if (int rc = e->launch_deferred_now()) return rc;
    workers->pending.erase(std::remove_if(workers->pending.begin(), workers->pending.end(),
                                          [this](Engine* e) { return e != this; }),
                           workers->pending.end());
    CK(cudaEventSynchronize(workers->last_done));
    CK(cudaStreamSynchronize(w.stream));
    CK(cudaStreamSynchronize(stream));
    if (!w.reserve(elem(), need[0], need[1], need[2], need[3], need[4], need[5], need[6]))
      return fail(this, 2, "sweep workspace allocation failed");
  }
  return 0;
}

template <typename C>
int Engine::run_sweep(SweepJob& job, SweepWork& w) {
  const SweepPlan& plan = *job.plan;
  const ShapeTrace& tr = job.tr;
  cudaStream_t s = w.stream;
  {
    size_t need[7] = {1, 1, 1, 256, 4, 16, 0};
    job_needs(job, need);
    if (w.elem != sizeof(C) || need[0] > w.cap_t || need[1] > w.cap_seg || need[2] > w.cap_x ||
        need[3] > w.svd_bytes || need[4] > w.nslots || need[5] > w.cap_d || need[6] > w.tc_bytes)
      return fail(this, 8, "sweep workspace was not reserved");
  }
  const C one = one_of<C>(), zero = zero_of<C>();
  auto slot = [&](int i) { return (C*)w.slot[i]; };
  C* Sb[2] = {(C*)w.S[0], (C*)w.S[1]};
  C* Rb[2] = {(C*)w.R[0], (C*)w.R[1]};
  C* qrA = (C*)w.qrA;
  C* qrQ = (C*)w.qrQ;
  C* qrR = (C*)w.qrR;
  C* tau = (C*)w.tau;

  std::vector<int> freelist;
  for (int i = (int)w.nslots - 1; i >= 0; --i) freelist.push_back(i);
  auto take = [&]() { int x = freelist.back(); freelist.pop_back(); return x; };
  auto give = [&](int x) { freelist.push_back(x); };
  std::vector<int> pos;
  std::vector<TShape> sh;
  long long launches = 0;

  CK(cudaMemsetAsync(w.logscale, 0, sizeof(double), s));
  CK(cudaMemsetAsync(w.status, 0, 2 * sizeof(int), s));
  pos.push_back(take());
  sh.push_back(TShape{1, 1, 1});
  CK(launch_fill(slot(pos.back()), 1, 1.0, 0.0, s));
  for (size_t q = 0; q < job.start.size(); ++q) {
    TShape t = job.start_shape[q];
    pos.push_back(take());
    CK(launch_copy_tensor((const C*)job.start[q], slot(pos.back()), t.l, t.p, t.r, plan.start_reversed, s));
    if (plan.start_reversed) std::swap(t.l, t.r);
    sh.push_back(t);
  }
  pos.push_back(take());
  sh.push_back(TShape{1, 1, 1});
  CK(launch_fill(slot(pos.back()), 1, 1.0, 0.0, s));
  launches += 2 + (long long)job.start.size();

  auto qr_move = [&](int c) -> int {   // centre c -> c + 1
    TShape a = sh[c], b = sh[c + 1];
    const int m = a.l * a.p, n = a.r, kk = std::min(m, n);
    CK(cudaMemcpyAsync(qrA, slot(pos[c]), sizeof(C) * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
    CK(launch_qr(qrA, m, n, qrQ, qrR, tau, s));
    CK(cudaMemcpyAsync(slot(pos[c]), qrQ, sizeof(C) * (size_t)m * kk, cudaMemcpyDeviceToDevice, s));
    sh[c].r = kk;
    const int t = take();
    CK(launch_zgemm('N', 'N', kk, b.p * b.r, n, one, qrR, n, 0, slot(pos[c + 1]), b.p * b.r, 0, zero, slot(t),
                    b.p * b.r, 0, 1, s));
    give(pos[c + 1]);
    pos[c + 1] = t;
    sh[c + 1].l = kk;
    launches += 4;
    return 0;
  };
  auto lq_move = [&](int c) -> int {   // centre c -> c - 1
    TShape b = sh[c], a = sh[c - 1];
    const int m = b.p * b.r, n = b.l, kk = std::min(m, n);
    CK(launch_conj_transpose(slot(pos[c]), b.l, b.p * b.r, qrA, s));
    CK(launch_qr(qrA, m, n, qrQ, qrR, tau, s));
    CK(launch_conj_transpose(qrQ, m, kk, slot(pos[c]), s));
    sh[c].l = kk;
    const int t = take();
    CK(launch_zgemm('N', 'C', a.l * a.p, kk, n, one, slot(pos[c - 1]), n, 0, qrR, n, 0, zero, slot(t), kk, 0, 1, s));
    give(pos[c - 1]);
    pos[c - 1] = t;
    sh[c - 1].r = kk;
    launches += 4;
    return 0;
  };
  auto normalise = [&](int c) -> int {
    CK(launch_normalise(slot(pos[c]), sh[c].size(), w.logscale, s));
    launches += 1;
    return 0;
  };

  for (int p = (int)pos.size() - 1; p >= 1; --p)
    if (int rc = lq_move(p)) return rc;
  int c = 0;
  if (int rc = normalise(0)) return rc;

  for (size_t si = 0; si < plan.steps.size(); ++si) {
    const SweepStep& st = plan.steps[si];
    const SweepNode& node = plan.nodes[st.node];
    const auto& rec = tr.steps[si];
    while (c < st.i) { if (int rc = qr_move(c)) return rc; ++c; }
    while (c > st.j) { if (int rc = lq_move(c)) return rc; --c; }
    const int l = sh[st.i].l, r = sh[st.j].r;
    const C* Sp;
    long long P;
    if (st.nin == 1) {
      Sp = slot(pos[st.i]);
      P = sh[st.i].p;
    } else {
      const C* cur = slot(pos[st.i]);
      long long rows = (long long)l * sh[st.i].p;
      int inner = sh[st.i].r;
      int buf = 0;
      for (int q = st.i + 1; q <= st.j; ++q) {
        const int cols = sh[q].p * sh[q].r;
        CK(merge_call((int)rows, cols, inner, cur, slot(pos[q]), Sb[buf], w.tc, w.tc_bytes, w.status + 1,
                      tc_mode != 0, s));
        cur = Sb[buf];
        buf ^= 1;
        rows *= sh[q].p;
        inner = sh[q].r;
        ++launches;
      }
      Sp = cur;
      P = rows / l;
    }
    if (P != rec.P) return fail(this, 8, "sweep: merged dimension disagrees with the plan");
    // contraction R[a, Q, b] = sum_P X[P, Q] S[a, P, b]
    const C* X = (const C*)job.node_tensor[st.node];
    if (node.site && !X) {             // K1 into the scratch, right before its use
      const auto& f = job.node_fuse[st.node];
      const double2* t = (const double2*)t_dev.p + (size_t)f[0] * d * D * D * D * D;
      const int perm[4] = {f[1], f[2], f[3], f[4]};
      CK(launch_fuse(t, d, D, site_n[f[0]].data(), nullptr, perm, (C*)w.X, s));
      X = (const C*)w.X;
      ++launches;
    } else if (!node.site) {
      const TShape ms = job.node_shape[st.node];
      int perm[3];
      for (int q = 0; q < st.nin; ++q) perm[q] = st.in_leg[q];
      for (int q = 0; q < st.nout; ++q) perm[st.nin + q] = st.out_leg[q];
      CK(launch_permute3(X, ms.l, ms.p, ms.r, perm, (C*)w.X, s));
      X = (const C*)w.X;
      ++launches;
    }
    const int Q = rec.Q;
    if (tc_mode && sizeof(C) == sizeof(float2)) {
      // split TF32 / BF16 on the tensor cores, FP32 accumulation
      CK(launch_tc_absorb(tc_mode == 2, X, (int)P, Q, Sp, l, r, Rb[0], w.tc, w.status + 1, s));
      launches += 6;
    } else {
      KTimerScope timer(KC_ABSORB, s, 8.0 * l * (double)P * Q * r);
      CK(launch_zgemm('T', 'N', Q, r, (int)P, one, X, Q, 0, Sp, r, P * r, zero, Rb[0], r, (long long)Q * r, l, s));
      ++launches;
    }
    sweep_flops += 8.0 * (double)l * (double)P * (double)Q * (double)r;
    std::vector<int> newpos;
    std::vector<TShape> newsh;
    if (st.nout == 0) {
      if (st.i > 0) {
        const TShape a = sh[st.i - 1];
        const int t = take();
        CK(launch_zgemm('N', 'N', a.l * a.p, r, l, one, slot(pos[st.i - 1]), l, 0, Rb[0], r, 0, zero, slot(t), r, 0,
                        1, s));
        give(pos[st.i - 1]);
        pos[st.i - 1] = t;
        sh[st.i - 1].r = r;
        for (int q = st.i; q <= st.j; ++q) give(pos[q]);
        pos.erase(pos.begin() + st.i, pos.begin() + st.j + 1);
        sh.erase(sh.begin() + st.i, sh.begin() + st.j + 1);
        c = st.i - 1;
      } else {
        const TShape b = sh[st.j + 1];
        const int t = take();
        CK(launch_zgemm('N', 'N', l, b.p * b.r, r, one, Rb[0], r, 0, slot(pos[st.j + 1]), b.p * b.r, 0, zero, slot(t),
                        b.p * b.r, 0, 1, s));
        give(pos[st.j + 1]);
        pos[st.j + 1] = t;
        sh[st.j + 1].l = l;
        for (int q = st.i; q <= st.j; ++q) give(pos[q]);
        pos.erase(pos.begin() + st.i, pos.begin() + st.j + 1);
        sh.erase(sh.begin() + st.i, sh.begin() + st.j + 1);
        c = st.i;
      }
      ++launches;
    } else {
      const C* cur = Rb[0];
      int rbuf = 1;
      int ll = l;
      long long rest = Q;
      for (int q = 0; q + 1 < st.nout; ++q) {
        const int q1 = rec.out_dims[q];
        rest /= q1;
        const int rows = ll * q1;
        const long long cols = rest * r;
        const int k = rec.split[q].r;
        const int t = take();
        const bool c64 = sizeof(C) == sizeof(float2);
        const int qsteps = c64 ? power_iters : power_iters64;
        // the range-finder products stay on the SIMT GEMM: their K is the
        // full split width (2304 at D = 6, chi = 64), where the tensor cores'
        // FP32 accumulation loses an order of magnitude against it
        CK(svd_call(cur, rows, (int)cols, chi, slot(t), Rb[rbuf], w.svd, w.status, s, qsteps, false, w.status + 1));
        launches += svd_launches(rows, (int)cols, chi, c64, qsteps);
        newpos.push_back(t);
        newsh.push_back(TShape{ll, q1, k});
        cur = Rb[rbuf];
        rbuf ^= 1;
        ll = k;
      }
      const int qlast = rec.out_dims[st.nout - 1];
      const int t = take();
      CK(cudaMemcpyAsync(slot(t), cur, sizeof(C) * (size_t)ll * qlast * r, cudaMemcpyDeviceToDevice, s));
      ++launches;
      newpos.push_back(t);
      newsh.push_back(TShape{ll, qlast, r});
      for (int q = st.i; q <= st.j; ++q) give(pos[q]);
      pos.erase(pos.begin() + st.i, pos.begin() + st.j + 1);
      sh.erase(sh.begin() + st.i, sh.begin() + st.j + 1);
      pos.insert(pos.begin() + st.i, newpos.begin(), newpos.end());
      sh.insert(sh.begin() + st.i, newsh.begin(), newsh.end());
      c = st.i + st.nout - 1;
    }
    if (int rc = normalise(c)) return rc;
  }
  const int n = (int)pos.size();
  if (plan.raw) {                      // a bubble halted before a core: the boundary as it stands
    if ((int)job.dest.size() != n || (int)tr.final_mps.size() != n)
      return fail(this, 8, "sweep: raw boundary length mismatch");
    for (int q = 0; q < n; ++q) {
      const TShape t = sh[q];
      const TShape f = tr.final_mps[q];
      if (t.l != f.l || t.p != f.p || t.r != f.r) return fail(this, 8, "sweep: raw boundary shape mismatch");
      CK(launch_copy_tensor(slot(pos[q]), (C*)job.dest[q], t.l, t.p, t.r, false, s));
      ++launches;
    }
    sweep_launches += launches;
    return 0;
  }
  if (n < 3) return fail(this, 8, "sweep: final boundary too short");
  {
    const int t = take();
    CK(launch_zgemm('N', 'N', 1, sh[1].p * sh[1].r, sh[0].r, one, slot(pos[0]), sh[0].r, 0, slot(pos[1]),
                    sh[1].p * sh[1].r, 0, zero, slot(t), sh[1].p * sh[1].r, 0, 1, s));
    give(pos[1]);
    pos[1] = t;
    sh[1].l = 1;
    const int t2 = take();
    const TShape b = sh[n - 2];
    CK(launch_zgemm('N', 'N', b.l * b.p, 1, b.r, one, slot(pos[n - 2]), b.r, 0, slot(pos[n - 1]), 1, 0, zero, slot(t2),
                    1, 0, 1, s));
    give(pos[n - 2]);
    pos[n - 2] = t2;
    sh[n - 2].r = 1;
    launches += 2;
  }
  const int L = n - 2;
  if (L != plan.out_len || (int)job.dest.size() != L) return fail(this, 8, "sweep: out face length mismatch");
  for (int q = 0; q < L; ++q) {
    const TShape t = sh[1 + q];
    const int di = plan.out_reversed ? (L - 1 - q) : q;
    CK(launch_copy_tensor(slot(pos[1 + q]), (C*)job.dest[di], t.l, t.p, t.r, plan.out_reversed, s));
    ++launches;
  }
  sweep_launches += launches;
  return 0;
}

// ------------------------------------------------------------ iteration
//
// One synchronous iteration (Alg. 1: every message update of the network
// from the current messages, then all replaced at once) runs on a private
// root stream: fork over the worker streams, one sweep and one finalisation
// per update, join, and the distances and statuses copied to pinned host
// memory.  iter_begin orders the root after the caller's stream, iter_end
// orders the caller's stream after the last iteration; in between any
// number of iter_launch / iter_finish pairs, which is what lets several
// contexts (bbp_batch_iterate, the server) keep iterations in flight at once.

int Engine::iter_begin() {
  DeviceScope ds(device);
  if (!partitioned) return fail(this, 8, "bbp_partition_blocks must come first");
  if (!messages_ready) return fail(this, 8, "bbp_init_messages must come first");
  const int nu = (int)geom.updates().size();
  // device: per-update distances, 2 status ints per update, tol, the word
  if (!dist_dev.ensure(sizeof(double) * nu + 2 * sizeof(int) * nu + 512, stream)) return fail(this, 2, "allocation failed");
  if (!h_word) CK(cudaHostAlloc((void**)&h_word, 4 * sizeof(double), cudaHostAllocDefault));
  if (!root) {
    CK(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&root_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&root_out, cudaEventDisableTiming));
  }
  CK(cudaEventRecord(root_in, stream));
  CK(cudaStreamWaitEvent(root, root_in, 0));
  return 0;
}

int Engine::iter_end() {
  DeviceScope ds(device);
  if (!root) return 0;
  CK(cudaEventRecord(root_out, root));
  CK(cudaStreamWaitEvent(stream, root_out, 0));
  return 0;
}

int Engine::iter_launch() {
  DeviceScope ds(device);
  std::lock_guard<std::mutex> lk(pool_ref().mu);
  return precision == 0 ? iter_launch_t<double2>() : iter_launch_t<float2>();
}

template <typename C>
int Engine::iter_launch_t() {
  const auto ups = geom.updates();
  const int nu = (int)ups.size();
  in_flight = false;
  if (nu == 0) return 0;
  int* status_dev = (int*)((double*)dist_dev.p + nu);
  double* tol_dev = (double*)((char*)dist_dev.p + ((sizeof(double) * nu + 2 * sizeof(int) * nu + 255) & ~size_t(255)));
  double* word_dev = tol_dev + 4;
  const int nstreams = std::max(1, std::min(nu, max_streams));
  for (int i = 0; i < nstreams; ++i)
    if (!work(i)) return fail(this, 3, "stream creation failed");
  CK(cudaStreamWaitEvent(root, workers->last_done, 0));   // the pool's previous user
  sweep_launches = 0;
  sweep_flops = 0.0;
  if (use_graphs) {
    // replay without rebuilding the jobs when nothing the graph reads changed
    const int par = 1 - msgs.at({ups[0].recv_block, ups[0].recv_face}).cur;
    IterGraph& g = graphs[par];
    if (g.graph && g.in_sig == input_signature(nstreams) && (int)g.out_shapes.size() == nu) {
      for (int u = 0; u < nu; ++u) msgs.at({ups[u].recv_block, ups[u].recv_face}).sh[par] = g.out_shapes[u];
      h_word[0] = iter_tol;
      sweep_launches = g.launches;
      sweep_flops = g.flops;
      launched_parity = par;
      launched_graph = true;
      in_flight = true;
      if (defer_graph) {
        pending_launch = true;
        workers->pending.push_back(this);
        return 0;
      }
      if (!g.exec) {
        const cudaError_t ce = cudaGraphInstantiate(&g.exec, g.graph, 0);
        if (ce != cudaSuccess) {
          in_flight = false;
          return fail(this, 3, std::string("graph instantiation: ") + cudaGetErrorString(ce));
        }
      }
      CK(cudaMemcpyAsync(tol_dev, h_word, sizeof(double), cudaMemcpyHostToDevice, root));
      CK(cudaGraphLaunch(g.exec, root));
      CK(cudaMemcpyAsync(h_word + 1, word_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, root));
      CK(cudaEventRecord(root_out, root));
      CK(cudaEventRecord(workers->last_done, root));
      return 0;
    }
  }
  std::vector<DBuf*> tmp;
  std::vector<SweepJob> jobs(nu);
  int rc = 0;
  for (int u = 0; u < nu && !rc; ++u) {
    const auto& up = ups[u];
    if ((rc = fill_job<C>(block_regions[up.block], plans.at({up.block, up.face}), jobs[u], {}, tmp))) break;
    Message& dst = msgs.at({up.recv_block, up.recv_face});
    for (const TShape& t : jobs[u].tr.final_mps)
      if ((size_t)t.size() > dst.cap) { rc = fail(this, 8, "message tensor exceeds its buffer"); break; }
  }
  for (DBuf* b : tmp) delete b;      // no operator insertions in an iteration
  if (rc) return rc;
  const unsigned long long in_sig = input_signature(nstreams);   // before the destinations change shape
  // destinations and their shapes (host bookkeeping, also when replaying)
  int parity = 0;
  for (int u = 0; u < nu; ++u) {
    const auto& up = ups[u];
    Message& dst = msgs.at({up.recv_block, up.recv_face});
    const int nxt = 1 - dst.cur;
    parity = nxt;
    jobs[u].dest.clear();
    for (int q = 0; q < dst.k(); ++q) jobs[u].dest.push_back(dst.tensor<C>(nxt, q));
    dst.sh[nxt] = jobs[u].tr.final_mps;
  }
  if ((rc = reserve_workers(jobs, nstreams))) return rc;
  if (learning())
    for (int u = 0; u < nu; ++u)
      if ((rc = reserve_learning(msgs.at({ups[u].recv_block, ups[u].recv_face})))) return rc;
  cudaEvent_t fork = root_in2;
  // fork onto the worker streams, one sweep and one finalisation per update, join
  auto enqueue = [&]() -> int {
    CK(cudaEventRecord(fork, root));
    for (int i = 0; i < nstreams; ++i) CK(cudaStreamWaitEvent(workers->w[i]->stream, fork, 0));
    int e = 0;
    for (int u = 0; u < nu && !e; ++u) {
      SweepWork& w = *workers->w[u % nstreams];
      const auto& up = ups[u];
      Message& dst = msgs.at({up.recv_block, up.recv_face});
      if ((e = run_sweep<C>(jobs[u], w))) break;
      if ((e = finalize_message<C>(dst, 1 - dst.cur, w, w.stream, (double*)dist_dev.p + u, true))) break;
      CK(cudaMemcpyAsync(status_dev + 2 * u, w.status, 2 * sizeof(int), cudaMemcpyDeviceToDevice, w.stream));
    }
    for (int i = 0; i < nstreams; ++i) {
      CK(cudaEventRecord(workers->w[i]->done, workers->w[i]->stream));
      CK(cudaStreamWaitEvent(root, workers->w[i]->done, 0));
    }
    if (!e) {
      CK(launch_iter_reduce((const double*)dist_dev.p, status_dev, nu, tol_dev, word_dev, root));
      sweep_launches += 1;
    }
    return e;
  };
  if (!root_in2) {
    CK(cudaEventCreateWithFlags(&root_in2, cudaEventDisableTiming));
    fork = root_in2;
  }
  // capture only once the inputs repeat: while the bond dimensions still
  // grow (the first iterations from bond-1 messages) every iteration would
  // need a new graph, and instantiating it costs more than launching eagerly
  h_word[0] = iter_tol;
  const bool stable = in_sig == last_in_sig[parity];
  last_in_sig[parity] = in_sig;
  const bool replayable = graphs[parity].graph && graphs[parity].sig == iter_signature(jobs, nstreams);
  launched_graph = use_graphs && (stable || replayable);
  if (!launched_graph || !defer_graph)
    CK(cudaMemcpyAsync(tol_dev, h_word, sizeof(double), cudaMemcpyHostToDevice, root));
  if (!launched_graph) {
    rc = enqueue();
  } else {
    IterGraph& g = graphs[parity];
    const unsigned long long sig = iter_signature(jobs, nstreams);
    if (!g.graph || g.sig != sig) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
      g = IterGraph();
      const long long tag = graph_tag(parity);
      ktimer_drop_tag(tag);
      ktimer_set_tag(tag);
      cudaError_t ce = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) {
        ktimer_set_tag(-1);
        return fail(this, 3, std::string("graph capture: ") + cudaGetErrorString(ce));
      }
      int e = enqueue();
      cudaGraph_t graph = nullptr;
      ce = cudaStreamEndCapture(root, &graph);
      ktimer_set_tag(-1);
      if (!e && ce != cudaSuccess) e = fail(this, 3, std::string("graph capture: ") + cudaGetErrorString(ce));
      if (!e && !defer_graph) {
        ce = cudaGraphInstantiate(&g.exec, graph, 0);
        if (ce != cudaSuccess) e = fail(this, 3, std::string("graph instantiation: ") + cudaGetErrorString(ce));
      }
      if (e) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (graph) cudaGraphDestroy(graph);
        g = IterGraph();
        return e;
      }
      g.graph = graph;
      g.uid = g_uid.fetch_add(1);
      g.sig = sig;
      g.launches = sweep_launches;
      g.flops = sweep_flops;
    }
    g.in_sig = in_sig;
    g.out_shapes.resize(nu);
    for (int u = 0; u < nu; ++u) g.out_shapes[u] = msgs.at({ups[u].recv_block, ups[u].recv_face}).sh[parity];
    sweep_launches = g.launches;
    sweep_flops = g.flops;
    if (defer_graph) {
      launched_parity = parity;
      in_flight = true;
      pending_launch = true;
      workers->pending.push_back(this);
      return 0;
    }
    if (!g.exec) {
      const cudaError_t ce = cudaGraphInstantiate(&g.exec, g.graph, 0);
      if (ce != cudaSuccess) return fail(this, 3, std::string("graph instantiation: ") + cudaGetErrorString(ce));
    }
    cudaError_t le = cudaGraphLaunch(g.exec, root);
    if (le != cudaSuccess) return fail(this, 3, std::string("graph launch: ") + cudaGetErrorString(le));
  }
  if (rc) return rc;
  CK(cudaMemcpyAsync(h_word + 1, word_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, root));
  CK(cudaEventRecord(root_out, root));
  CK(cudaEventRecord(workers->last_done, root));
  launched_parity = parity;
  in_flight = true;
  return 0;
}

int Engine::iter_finish(double* err_out) {
  DeviceScope ds(device);
  const auto ups = geom.updates();
  const int nu = (int)ups.size();
  if (nu == 0) {
    if (err_out) *err_out = 0.0;
    return 0;
  }
  if (!in_flight) return fail(this, 8, "no iteration in flight");
  if (pending_launch) {
    in_flight = false;
    pending_launch = false;
    if (workers) {
      std::lock_guard<std::mutex> lk(workers->mu);
      auto& pv = workers->pending;
      pv.erase(std::remove(pv.begin(), pv.end(), this), pv.end());
    }
    return fail(this, 8, "a deferred iteration was never launched");
  }
  in_flight = false;
  CK(cudaEventSynchronize(root_out));
  if (ktimer_class()) ktimer_collect(launched_graph ? graph_tag(launched_parity) : -1);
  // the convergence word of the iteration (k_iter_reduce)
  const double err = h_word[1];
  int flags = 0;
  std::memcpy(&flags, h_word + 2, sizeof(int));
  const bool nonfinite = flags & 1, sweep_limit = flags & 2, tc_timeout = flags & 4;
  last_converged = (flags & 8) != 0;
  for (const auto& up : ups) msgs.at({up.recv_block, up.recv_face}).cur ^= 1;
  launches_per_iter = sweep_launches;
  flops_per_iter = sweep_flops;
  ++n_iterations;
  if (err_out) *err_out = err;
  if (tc_timeout) return fail(this, 7, "a tensor-core pipeline wait timed out");
  if (nonfinite || sweep_limit)
    return fail(this, 5, nonfinite ? "a message became non-finite" : "a Jacobi SVD reached its sweep limit");
  return 0;
}

int Engine::iterate(double tol, int max_iter, int* iters, double* err_out) {
  if (max_iter < 0 || !(tol >= 0.0)) return fail(this, 1, "tol must be >= 0 and max_iter >= 0");
  iter_tol = tol;
  int rc = iter_begin();
  if (rc) return rc;
  double err = geom.updates().empty() ? 0.0 : INFINITY;
  int it = 0;
  for (; it < max_iter && !geom.updates().empty(); ++it) {
    if ((rc = iter_launch())) break;
    rc = iter_finish(&err);
    if (rc) { ++it; break; }
    if (last_converged) { ++it; break; }   // the device's convergence word
  }
  const int rc2 = iter_end();
  if (iters) *iters = it;
  if (err_out) *err_out = err;
  if (rc) return rc;
  if (rc2) return rc2;
  if (err > tol) return fail(this, 6, "max_iter reached before the messages converged");
  return 0;
}

// --------------------------------------------------------------- observables

int Engine::contract_batch(const std::vector<std::vector<std::array<int, 2>>>& coords, const std::vector<OpList>& ops,
                           std::vector<double>& logscale, std::vector<double>& re, std::vector<double>& im) {
  return precision == 0 ? contract_batch_t<double2>(coords, ops, logscale, re, im)
                        : contract_batch_t<float2>(coords, ops, logscale, re, im);
}

template <typename C>
int Engine::contract_batch_t(const std::vector<std::vector<std::array<int, 2>>>& coords, const std::vector<OpList>& ops,
                             std::vector<double>& logscale, std::vector<double>& re, std::vector<double>& im) {
  if (!partitioned || !messages_ready) return fail(this, 8, "partition and messages are required first");
  const int nj = (int)coords.size();
  logscale.assign(nj, 0.0);
  re.assign(nj, 0.0);
  im.assign(nj, 0.0);
  const int nstreams = std::max(1, std::min(nj, 16));
  std::lock_guard<std::mutex> lk(pool_ref().mu);
  for (int i = 0; i < nstreams; ++i)
    if (!work(i)) return fail(this, 3, "stream creation failed");
  CK(cudaStreamWaitEvent(stream, workers->last_done, 0));   // the pool's previous user
  cudaEvent_t fork;
  CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  DBuf res;
  if (!res.ensure(sizeof(double) * 4 * nj + 256, stream)) return fail(this, 2, "allocation failed");
  std::vector<DBuf*> tmp;
  int rc = 0;
  std::vector<Region> regions(nj);
  std::vector<SweepPlan> plansv(nj);
  std::vector<SweepJob> jobs(nj);
  for (int j = 0; j < nj && !rc; ++j) {
    std::string err = build_region(geom, coords[j], regions[j]);
    if (!err.empty()) { rc = fail(this, 1, err); break; }
    err = compile_sweep(geom, regions[j], TOP, plansv[j]);
    if (!err.empty()) { rc = fail(this, 8, "sweep plan: " + err); break; }
    SweepJob& job = jobs[j];
    if ((rc = fill_job<C>(regions[j], plansv[j], job, ops[j], tmp))) break;
    DBuf* out = new DBuf();
    tmp.push_back(out);
    size_t tot = 0;
    for (const TShape& t : job.tr.final_mps) tot += (size_t)t.size();
    if (!out->ensure(sizeof(C) * tot + 256, stream)) { rc = fail(this, 2, "allocation failed"); break; }
    size_t off = 0;
    job.dest.clear();
    for (const TShape& t : job.tr.final_mps) { job.dest.push_back((C*)out->p + off); off += (size_t)t.size(); }
  }
  if (!rc) rc = reserve_workers(jobs, nstreams);
  if (!rc) {
    CK(cudaEventRecord(fork, stream));
    for (int i = 0; i < nstreams; ++i) CK(cudaStreamWaitEvent(workers->w[i]->stream, fork, 0));
  }
  for (int j = 0; j < nj && !rc; ++j) {
    SweepWork& w = *workers->w[j % nstreams];
    SweepJob& job = jobs[j];
    if ((rc = run_sweep<C>(job, w))) break;
    ChainDesc A{}, B{};
    for (size_t q = 0; q < job.dest.size() && q < (size_t)kMaxChain; ++q) {
      const TShape t = job.tr.final_mps[q];
      A.T[A.k] = job.dest[q];
      A.l[A.k] = t.l; A.p[A.k] = t.p; A.r[A.k] = t.r;
      ++A.k;
    }
    for (const auto& f : regions[j].side_faces[TOP]) {
      const Message& m = msgs.at({regions[j].ids[f[0]], f[1]});
      for (int q = 0; q < m.k() && B.k < kMaxChain; ++q) {
        const TShape t = m.sh[m.cur][q];
        B.T[B.k] = m.tensor<C>(m.cur, q);
        B.l[B.k] = t.l; B.p[B.k] = t.p; B.r[B.k] = t.r;
        ++B.k;
      }
    }
    if (A.k != B.k || job.dest.size() > (size_t)kMaxChain) { rc = fail(this, 8, "top face mismatch"); break; }
    CK(launch_mps_dot(A, B, sizeof(C) == sizeof(float2), w.k4, w.scal, w.stream));
    double* rp = (double*)res.p + 4 * j;
    CK(cudaMemcpyAsync(rp, w.logscale, sizeof(double), cudaMemcpyDeviceToDevice, w.stream));
    CK(cudaMemcpyAsync(rp + 1, w.scal, sizeof(double2), cudaMemcpyDeviceToDevice, w.stream));
    CK(cudaMemcpyAsync(rp + 3, w.status, sizeof(int), cudaMemcpyDeviceToDevice, w.stream));
  }
  for (int i = 0; i < nstreams; ++i) {
    CK(cudaEventRecord(workers->w[i]->done, workers->w[i]->stream));
    CK(cudaStreamWaitEvent(stream, workers->w[i]->done, 0));
  }
  CK(cudaEventRecord(workers->last_done, stream));
  std::vector<double> h(4 * (size_t)nj);
  if (!rc) CK(cudaMemcpyAsync(h.data(), res.p, sizeof(double) * 4 * nj, cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  for (DBuf* b : tmp) delete b;
  cudaEventDestroy(fork);
  if (rc) return rc;
  for (int j = 0; j < nj; ++j) {
    logscale[j] = h[4 * j];
    re[j] = h[4 * j + 1];
    im[j] = h[4 * j + 2];
    int st;
    std::memcpy(&st, &h[4 * j + 3], sizeof(int));
    if (st != 0) return fail(this, 5, "an SVD did not converge in a contraction");
  }
  return 0;
}

int Engine::bond_region(int g1, int k1, std::vector<std::array<int, 2>>& coords, std::array<int, 2>& key1,
                        std::array<int, 2>& key2) {
  int loc = -1;
  int bid = geom.home_block(g1, &loc);
  if (bid < 0 || k1 < 0 || k1 > 3) return fail(this, 1, "site or slot out of range");
  const Block& b = geom.blocks[bid];
  int t = b.sites[loc][0], i = b.sites[loc][1], j = b.sites[loc][2];
  int t2, i2, j2, k2;
  geom.lat.neighbour(t, i, j, k1, t2, i2, j2, k2);
  if (geom.lat.site_id(t2, i2, j2) < 0) return fail(this, 1, "the slot points out of an open lattice");
  int X2, Y2;
  geom.block_of(t2, i2, j2, X2, Y2);
  key1 = {0, loc};
  if (X2 == b.X && Y2 == b.Y) {
    coords = {{b.X, b.Y}};
    key2 = {0, b.local_of(t2, i2, j2)};
    return 0;
  }
  coords = {{b.X, b.Y}, {X2, Y2}};
  const Block& b2 = geom.blocks[geom.block_id(X2, Y2)];
  key2 = {1, b2.local_of(t2, i2 - (X2 - b2.X) * geom.bx, j2 - (Y2 - b2.Y) * geom.by)};
  if (key2[1] < 0) return fail(this, 8, "neighbour not found in its block");
  return 0;
}

// <S_i . S_j> of the given bonds (site, slot): per bond the region of
// reading E contracted with nothing inserted and with S^a (x) S^a for
// a = x, y, z, all contractions of all bonds in one batch.
int Engine::bond_energies(const std::vector<std::array<int, 2>>& bonds, std::vector<double>& out) {
  if (d != 2) return fail(this, 1, "the Heisenberg energy needs d = 2");
  static const double sx[8] = {0, 0, 0.5, 0, 0.5, 0, 0, 0};
  static const double sy[8] = {0, 0, 0, -0.5, 0, 0.5, 0, 0};
  static const double sz[8] = {0.5, 0, 0, 0, 0, 0, -0.5, 0};
  if (!op_dev.ensure(sizeof(double) * 24, stream)) return fail(this, 2, "allocation failed");
  double hops[24];
  std::memcpy(hops, sx, sizeof(sx));
  std::memcpy(hops + 8, sy, sizeof(sy));
  std::memcpy(hops + 16, sz, sizeof(sz));
  CK(cudaMemcpyAsync(op_dev.p, hops, sizeof(hops), cudaMemcpyHostToDevice, stream));
  const double* dsx = (const double*)op_dev.p;
  std::vector<std::vector<std::array<int, 2>>> Cc;
  std::vector<OpList> O;
  for (const auto& bk : bonds) {
    if (bk[0] < 0 || bk[0] >= geom.lat.n_sites() || bk[1] < 0 || bk[1] > 3) return fail(this, 1, "bond out of range");
    std::vector<std::array<int, 2>> coords;
    std::array<int, 2> k1, k2;
    if (int rc = bond_region(bk[0], bk[1], coords, k1, k2)) return rc;
    Cc.push_back(coords);
    O.push_back({});
    for (const double* op : {dsx, dsx + 8, dsx + 16}) {
      Cc.push_back(coords);
      O.push_back({{k1, op}, {k2, op}});
    }
  }
  std::vector<double> ls, re, im;
  if (int rc = contract_batch(Cc, O, ls, re, im)) return rc;
  out.assign(bonds.size(), 0.0);
  for (size_t b = 0; b < bonds.size(); ++b) {
    const size_t j0 = 4 * b;
    double tot = 0.0;
    for (int a = 1; a <= 3; ++a) {
      const double r0 = re[j0], i0 = im[j0], r1 = re[j0 + a], i1 = im[j0 + a];
      tot += std::exp(ls[j0 + a] - ls[j0]) * (r1 * r0 + i1 * i0) / (r0 * r0 + i0 * i0);
    }
    out[b] = tot;
  }
  return 0;
}

int Engine::energy_per_site(double* e) {
  if (d != 2) return fail(this, 1, "the Heisenberg energy needs d = 2");
  static const double sx[8] = {0, 0, 0.5, 0, 0.5, 0, 0, 0};
  static const double sy[8] = {0, 0, 0, -0.5, 0, 0.5, 0, 0};
  static const double sz[8] = {0.5, 0, 0, 0, 0, 0, -0.5, 0};
  if (!op_dev.ensure(sizeof(double) * 24, stream)) return fail(this, 2, "allocation failed");
  double hops[24];
  std::memcpy(hops, sx, sizeof(sx));
  std::memcpy(hops + 8, sy, sizeof(sy));
  std::memcpy(hops + 16, sz, sizeof(sz));
  CK(cudaMemcpyAsync(op_dev.p, hops, sizeof(hops), cudaMemcpyHostToDevice, stream));
  const double* dsx = (const double*)op_dev.p;
  const double* dsy = dsx + 8;
  const double* dsz = dsx + 16;
  std::vector<std::vector<std::array<int, 2>>> Cc;
  std::vector<OpList> O;
  const Lattice& L = geom.lat;
  std::vector<std::array<int, 4>> seen;
  int nb = 0;
  for (int j = 0; j < L.Ly; ++j)
    for (int i = 0; i < L.Lx; ++i)
      for (int t = 0; t < L.ntypes(); ++t) {
        int g = L.site_id(t, i, j);
        for (int k = 0; k < 4; ++k) {
          int t2, i2, j2, k2;
          L.neighbour(t, i, j, k, t2, i2, j2, k2);
          int g2 = L.site_id(t2, i2, j2);
          if (g2 < 0) continue;
          std::array<int, 4> key = {g, k, g2, k2};
          std::array<int, 4> rev = {g2, k2, g, k};
          if (std::find(seen.begin(), seen.end(), rev) != seen.end()) continue;
          seen.push_back(key);
          std::vector<std::array<int, 2>> coords;
          std::array<int, 2> k1, kk2;
          if (int rc = bond_region(g, k, coords, k1, kk2)) return rc;
          Cc.push_back(coords);
          O.push_back({});
          for (const double* op : {dsx, dsy, dsz}) {
            Cc.push_back(coords);
            O.push_back({{k1, op}, {kk2, op}});
          }
          ++nb;
        }
      }
  std::vector<double> ls, re, im;
  if (int rc = contract_batch(Cc, O, ls, re, im)) return rc;
  double tot = 0.0;
  for (int b = 0; b < nb; ++b) {
    const int j0 = 4 * b;
    for (int a = 1; a <= 3; ++a) {
      double r0 = re[j0], i0 = im[j0], r1 = re[j0 + a], i1 = im[j0 + a];
      double den = r0 * r0 + i0 * i0;
      double scale = std::exp(ls[j0 + a] - ls[j0]);
      tot += scale * (r1 * r0 + i1 * i0) / den;
    }
  }
  *e = tot / L.n_sites();
  return 0;
}

int Engine::log_norm(double* out) { return precision == 0 ? log_norm_t<double2>(out) : log_norm_t<float2>(out); }

template <typename C>
int Engine::log_norm_t(double* out) {
  std::vector<std::vector<std::array<int, 2>>> Cc;
  std::vector<OpList> O;
  for (const Block& b : geom.blocks) {
    Cc.push_back({{b.X, b.Y}});
    O.push_back({});
  }
  std::vector<double> ls, re, im;
  if (int rc = contract_batch(Cc, O, ls, re, im)) return rc;
  double total = 0.0;
  for (size_t b = 0; b < Cc.size(); ++b) total += ls[b] + 0.5 * std::log(re[b] * re[b] + im[b] * im[b]);
  SweepWork* w = work(0);
  if (!w || !w->reserve(sizeof(C), 16, 16, 16, 4096, 4, 16, 0)) return fail(this, 2, "allocation failed");
  std::vector<std::pair<std::pair<int, int>, std::pair<int, int>>> pairs;
  for (const auto& u : geom.updates()) {
    auto a = std::make_pair(u.block, u.face), r = std::make_pair(u.recv_block, u.recv_face);
    bool dup = false;
    for (auto& pr : pairs) dup = dup || (pr.first == r && pr.second == a);
    if (!dup) pairs.push_back({a, r});
  }
  for (auto& pr : pairs) {
    const Message& m1 = msgs.at(pr.first);
    const Message& m2 = msgs.at(pr.second);
    CK(launch_mps_dot(chain_of<C>(m1, m1.cur), chain_of<C>(m2, m2.cur), sizeof(C) == sizeof(float2), w->k4, w->scal,
                      stream));
    double2 v;
    CK(cudaMemcpyAsync(&v, w->scal, sizeof(double2), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    total -= 0.5 * std::log(v.x * v.x + v.y * v.y);
  }
  *out = total;
  return 0;
}

int Engine::get_message(int block, int face, int* k, int* shapes, double* data, size_t cap) {
  return precision == 0 ? get_message_t<double2>(block, face, k, shapes, data, cap)
                        : get_message_t<float2>(block, face, k, shapes, data, cap);
}

template <typename C>
int Engine::get_message_t(int block, int face, int* k, int* shapes, double* data, size_t cap) {
  auto it = msgs.find({block, face});
  if (it == msgs.end()) return fail(this, 1, "no such message");
  const Message& m = it->second;
  if (!messages_ready) return fail(this, 8, "messages are not initialised");
  if (m.k() > 64) return fail(this, 1, "message too long");
  size_t need = 0;
  for (int q = 0; q < m.k(); ++q) need += 2 * (size_t)m.sh[m.cur][q].size();
  if (need > cap) return fail(this, 1, "output buffer too small");
  *k = m.k();
  size_t off = 0;
  std::vector<C> tmp;
  for (int q = 0; q < m.k(); ++q) {
    const TShape t = m.sh[m.cur][q];
    shapes[3 * q] = t.l;
    shapes[3 * q + 1] = t.p;
    shapes[3 * q + 2] = t.r;
    tmp.resize(t.size());
    CK(cudaMemcpyAsync(tmp.data(), m.tensor<C>(m.cur, q), sizeof(C) * t.size(), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    for (long long e = 0; e < t.size(); ++e) {
      data[off + 2 * e] = tmp[e].x;
      data[off + 2 * e + 1] = tmp[e].y;
    }
    off += 2 * (size_t)t.size();
  }
  return 0;
}

// ------------------------------------------------------------ core (Sec. 2.3)
//
// Two bubbles approach the core from the bottom and top faces of the block:
// the bottom-up bubble swallows every node before the core's last site (in
// the bottom-up sweep order), the top-down bubble every node after it; both
// skip the core, truncate like the message update, and return their
// boundary as it stands (raw plans).  The bubbles share their two end bonds
// and the legs of the two front lines; the zipper contracts each front line
// into one matrix (E_L on the left, E_R on the right), which is folded into
// the last tensor of the bottom bubble's core segment (E_R) and of the top
// bubble's (E_L^T).  What is left is the periodic MPS around the core: the
// bottom bubble's core legs left to right, then the top bubble's right to
// left, the last tensor's right bond closing onto the first one's left bond.

// The ring of one core on the device: the two bubbles' boundaries (outb),
// the folded tensors (fold), and per pMPS tensor its device pointer and
// shape.  The destructor waits for the work queued on the buffers.
template <typename C>
struct CoreRing {
  Engine* e = nullptr;
  DBuf outb[2], res, scratch, fold;    // res: [0..1] log scales, [2..3] status words of the bubbles
  CorePlan cp;
  std::vector<const C*> t;
  std::vector<TShape> sh;
  ~CoreRing() {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    for (size_t i = 0; e->workers && i < 2 && i < e->workers->w.size(); ++i)
      cudaStreamSynchronize(e->workers->w[i]->stream);
  }
};

template <typename C>
int Engine::core_ring(int block, const std::vector<int>& core, CoreRing<C>& ring) {
  ring.e = this;
  if (!partitioned || !messages_ready) return fail(this, 8, "partition and messages are required first");
  if (block < 0 || block >= (int)geom.blocks.size()) return fail(this, 1, "block out of range");
  const Region& R = block_regions[block];
  CorePlan& cp = ring.cp;
  const std::string err = compile_core(geom, R, core, cp);
  if (!err.empty()) return fail(this, 1, "core: " + err);
  const SweepPlan& pb = cp.bottom;
  const SweepPlan& pt = cp.top;
  const int n = (int)pb.final_labels.size(), m = (int)pt.final_labels.size();
  const int a = cp.a, c = cp.c;

  std::vector<DBuf*> tmp;
  struct TmpGuard {
    std::vector<DBuf*>& v;
    ~TmpGuard() { for (DBuf* b : v) delete b; }
  } guard{tmp};
  std::vector<SweepJob> jobs(2);
  if (int rc = fill_job<C>(R, pb, jobs[0], {}, tmp)) return rc;
  if (int rc = fill_job<C>(R, pt, jobs[1], {}, tmp)) return rc;
  if ((int)jobs[0].tr.final_mps.size() != n || (int)jobs[1].tr.final_mps.size() != m)
    return fail(this, 8, "core bubbles: boundary length disagrees with the plan");
  for (int j = 0; j < 2; ++j) {
    size_t tot = 0;
    for (const TShape& t : jobs[j].tr.final_mps) tot += (size_t)t.size();
    if (!ring.outb[j].ensure(sizeof(C) * tot + 256, stream)) return fail(this, 2, "allocation failed");
    size_t off = 0;
    jobs[j].dest.clear();
    for (const TShape& t : jobs[j].tr.final_mps) {
      jobs[j].dest.push_back((C*)ring.outb[j].p + off);
      off += (size_t)t.size();
    }
  }
  if (!ring.res.ensure(4 * sizeof(double) + 256, stream)) return fail(this, 2, "allocation failed");
  {
    std::lock_guard<std::mutex> lk(pool_ref().mu);
    for (int i = 0; i < 2; ++i)
      if (!work(i)) return fail(this, 3, "stream creation failed");
    CK(cudaStreamWaitEvent(stream, workers->last_done, 0));   // the pool's previous user
    if (int rc = reserve_workers(jobs, 2)) return rc;
    cudaEvent_t fork;
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    struct EvGuard {
      cudaEvent_t e;
      ~EvGuard() { cudaEventDestroy(e); }
    } eg{fork};
    CK(cudaEventRecord(fork, stream));
    for (int i = 0; i < 2; ++i) {
      SweepWork& w = *workers->w[i];
      CK(cudaStreamWaitEvent(w.stream, fork, 0));
      if (int rc = run_sweep<C>(jobs[i], w)) return rc;
      double* rp = (double*)ring.res.p;
      CK(cudaMemcpyAsync(rp + i, w.logscale, sizeof(double), cudaMemcpyDeviceToDevice, w.stream));
      CK(cudaMemcpyAsync(rp + 2 + i, w.status, 2 * sizeof(int), cudaMemcpyDeviceToDevice, w.stream));
      CK(cudaEventRecord(w.done, w.stream));
      CK(cudaStreamWaitEvent(stream, w.done, 0));
    }
    CK(cudaEventRecord(workers->last_done, stream));
  }

  // the zipper, on the context's stream (operands in outb and private scratch)
  const std::vector<TShape>& SB = jobs[0].tr.final_mps;
  const std::vector<TShape>& ST = jobs[1].tr.final_mps;
  const std::vector<void*> dB = jobs[0].dest, dT = jobs[1].dest;
  auto Bq = [&](int q) { return (const C*)dB[q]; };
  auto Tq = [&](int q) { return (const C*)dT[q]; };
  size_t mb = 1, mt = 1, mp = 1, mT = 1;
  for (const TShape& t : SB) { mb = std::max<size_t>(mb, std::max(t.l, t.r)); mp = std::max<size_t>(mp, t.p); }
  for (const TShape& t : ST) {
    mt = std::max<size_t>(mt, std::max(t.l, t.r));
    mp = std::max<size_t>(mp, t.p);
    mT = std::max<size_t>(mT, (size_t)t.size());
  }
  const size_t capE = mb * mt, capF = mb * mp * mt;
  if (!ring.scratch.ensure(sizeof(C) * (4 * capE + capF + mT) + 256, stream)) return fail(this, 2, "allocation failed");
  C* EL = (C*)ring.scratch.p;
  C* ER = EL + capE;
  C* Ea = ER + capE;
  C* Eb = Ea + capE;
  C* F = Eb + capE;
  C* Pm = F + capF;
  const C one = one_of<C>(), zero = zero_of<C>();
  // left front line: E[x, y] (x a bond of the bottom bubble, y of the top one)
  int ex = 1, ey = 1;
  CK(launch_fill(Ea, 1, 1.0, 0.0, stream));
  for (int q = 0; q < a; ++q) {
    const TShape b = SB[q], t = ST[m - 1 - q];
    if (b.l != ex || t.r != ey || b.p != t.p) return fail(this, 8, "zipper: shapes do not match");
    // F[y, (p z)] = sum_x E[x, y] B[x, (p z)]
    CK(launch_zgemm('T', 'N', ey, b.p * b.r, ex, one, Ea, ey, 0, Bq(q), b.p * b.r, 0, zero, F, b.p * b.r, 0, 1, stream));
    const int perm[3] = {2, 1, 0};   // T[w, p, y] -> [y, p, w]
    CK(launch_permute3(Tq(m - 1 - q), t.l, t.p, t.r, perm, Pm, stream));
    // E'[z, w] = sum_{(y p)} F[(y p), z] P[(y p), w]
    CK(launch_zgemm('T', 'N', b.r, t.l, ey * b.p, one, F, b.r, 0, Pm, t.l, 0, zero, Eb, t.l, 0, 1, stream));
    std::swap(Ea, Eb);
    ex = b.r;
    ey = t.l;
  }
  const int elx = ex, ely = ey;
  CK(cudaMemcpyAsync(EL, Ea, sizeof(C) * (size_t)ex * ey, cudaMemcpyDeviceToDevice, stream));
  // right front line: E[z, w] from the right ends inwards
  ex = 1;
  ey = 1;
  CK(launch_fill(Ea, 1, 1.0, 0.0, stream));
  for (int q = 0; q < c; ++q) {
    const TShape b = SB[n - 1 - q], t = ST[q];
    if (b.r != ex || t.l != ey || b.p != t.p) return fail(this, 8, "zipper: shapes do not match");
    // G[(x p), w] = sum_z B[(x p), z] E[z, w]
    CK(launch_zgemm('N', 'N', b.l * b.p, ey, ex, one, Bq(n - 1 - q), ex, 0, Ea, ey, 0, zero, F, ey, 0, 1, stream));
    const int perm[3] = {1, 0, 2};   // T[w, p, y] -> [p, w, y]
    CK(launch_permute3(Tq(q), t.l, t.p, t.r, perm, Pm, stream));
    // E'[x, y] = sum_{(p w)} G[x, (p w)] P[(p w), y]
    CK(launch_zgemm('N', 'N', b.l, t.r, b.p * ey, one, F, b.p * ey, 0, Pm, t.r, 0, zero, Eb, t.r, 0, 1, stream));
    std::swap(Ea, Eb);
    ex = b.l;
    ey = t.r;
  }
  const int erx = ex, ery = ey;
  CK(cudaMemcpyAsync(ER, Ea, sizeof(C) * (size_t)ex * ey, cudaMemcpyDeviceToDevice, stream));

  // the pMPS: B[a .. n-c-1] (the last times E_R), then T[c .. m-a-1] (the last times E_L^T)
  const int kb = n - c - 1, kt = m - a - 1;
  if (SB[kb].r != erx || ST[c].l != ery || ST[kt].r != ely || SB[a].l != elx)
    return fail(this, 8, "zipper: the ring does not close");
  const size_t fb = (size_t)SB[kb].l * SB[kb].p * ery, ft = (size_t)ST[kt].l * ST[kt].p * elx;
  if (!ring.fold.ensure(sizeof(C) * (fb + ft) + 256, stream)) return fail(this, 2, "allocation failed");
  C* FB = (C*)ring.fold.p;
  C* FT = FB + fb;
  CK(launch_zgemm('N', 'N', SB[kb].l * SB[kb].p, ery, erx, one, Bq(kb), erx, 0, ER, ery, 0, zero, FB, ery, 0, 1,
                  stream));
  CK(launch_zgemm('N', 'T', ST[kt].l * ST[kt].p, elx, ely, one, Tq(kt), ely, 0, EL, ely, 0, zero, FT, elx, 0, 1,
                  stream));
  ring.t.clear();
  ring.sh.clear();
  for (const auto& rq : cp.ring) {
    const int q = rq[1];
    if (rq[0] == 0) {
      TShape t = SB[q];
      if (q == kb) t.r = ery;
      ring.t.push_back(q == kb ? FB : Bq(q));
      ring.sh.push_back(t);
    } else {
      TShape t = ST[q];
      if (q == kt) t.r = elx;
      ring.t.push_back(q == kt ? FT : Tq(q));
      ring.sh.push_back(t);
    }
  }
  const int L = (int)ring.sh.size();
  for (int q = 0; q < L; ++q)
    if (ring.sh[q].r != ring.sh[(q + 1) % L].l) return fail(this, 8, "zipper: pMPS bonds do not close");
  return 0;
}

// log scales and statuses of the two bubbles (synchronises the stream)
template <typename C>
int Engine::core_ring_result(CoreRing<C>& ring, double* logscale) {
  double hres[4];
  CK(cudaMemcpyAsync(hres, ring.res.p, sizeof(hres), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  int st[4];
  std::memcpy(&st[0], &hres[2], 2 * sizeof(int));
  std::memcpy(&st[2], &hres[3], 2 * sizeof(int));
  if (st[1] || st[3]) return fail(this, 7, "a tensor-core wait timed out in a core bubble");
  if (st[0] || st[2]) return fail(this, 5, "an SVD did not converge in a core bubble");
  *logscale = hres[0] + hres[1];
  return 0;
}

int Engine::core_pmps(int block, const std::vector<int>& core, std::vector<TShape>& shapes,
                      std::vector<std::array<int, 2>>& legs, std::vector<double2>& data, double* logscale) {
  DeviceScope ds(device);
  return precision == 0 ? core_pmps_t<double2>(block, core, shapes, legs, data, logscale)
                        : core_pmps_t<float2>(block, core, shapes, legs, data, logscale);
}

template <typename C>
int Engine::core_pmps_t(int block, const std::vector<int>& core, std::vector<TShape>& shapes,
                        std::vector<std::array<int, 2>>& legs, std::vector<double2>& data, double* logscale) {
  CoreRing<C> ring;
  if (int rc = core_ring<C>(block, core, ring)) return rc;
  shapes = ring.sh;
  legs = ring.cp.legs;
  size_t tot = 0;
  for (const TShape& t : ring.sh) tot += (size_t)t.size();
  std::vector<C> host(tot);
  size_t off = 0;
  for (size_t q = 0; q < ring.t.size(); ++q) {
    CK(cudaMemcpyAsync(host.data() + off, ring.t[q], sizeof(C) * (size_t)ring.sh[q].size(), cudaMemcpyDeviceToHost,
                       stream));
    off += (size_t)ring.sh[q].size();
  }
  if (int rc = core_ring_result<C>(ring, logscale)) return rc;
  data.resize(tot);
  for (size_t e = 0; e < tot; ++e) data[e] = make_double2((double)host[e].x, (double)host[e].y);
  return 0;
}

// Local quantities of the core (Sec. 2.3, "Edge"): the ring is cut into two
// runs, A (bonds l0 -> m, legs' product P1) and B (m -> l0, product P2).  A
// bond core: A holds site 0's legs, B site 1's; with the fused site tensors
// laid out as [outer legs in ring order, joint leg],
// Z(O) = sum_{l0, m, j} (A T1(O1))[l0, m, j] (B T2(O2))[l0, m, j].
// A one-site core: A and B each hold half of its legs, T1 = [first half,
// second half], and Z(O) = sum_{l0, m, j} (A T1(O))[l0, m, j] B[l0, m, j].
int Engine::core_expect(int block, const std::vector<int>& core, const double* ops, int nops, double* re, double* im) {
  DeviceScope ds(device);
  return precision == 0 ? core_expect_t<double2>(block, core, ops, nops, re, im)
                        : core_expect_t<float2>(block, core, ops, nops, re, im);
}

template <typename C>
int Engine::core_expect_t(int block, const std::vector<int>& core, const double* ops, int nops, double* re,
                          double* im) {
  const int nc = (int)core.size();
  if (nc < 1 || nc > 2) return fail(this, 1, "core observables need one site or the two ends of a bond");
  if (nops < 0 || (nops > 0 && !ops)) return fail(this, 1, "bad operator list");
  CoreRing<C> ring;
  if (int rc = core_ring<C>(block, core, ring)) return rc;
  const Region& R = block_regions[block];
  const RSite* rs[2] = {nullptr, nullptr};
  for (int q = 0; q < nc; ++q)
    for (const RSite& x : R.sites)
      if (x.inst == 0 && x.local == core[q]) rs[q] = &x;
  if (!rs[0] || (nc == 2 && !rs[1])) return fail(this, 8, "core site missing from the block region");
  int js[2] = {-1, -1}, njoint = 0;
  if (nc == 2)
    for (int s1 = 0; s1 < 4; ++s1)
      for (int s2 = 0; s2 < 4; ++s2)
        if (rs[0]->label[s1] == rs[1]->label[s2]) { js[0] = s1; js[1] = s2; ++njoint; }
  if (nc == 2 && njoint != 1) return fail(this, 1, "the two core sites must share exactly one bond");
  // ring order starting at site 0's run of legs
  const auto& legs = ring.cp.legs;
  const int L = (int)legs.size();
  int start = 0;
  if (nc == 2) {
    start = -1;
    for (int q = 0; q < L && start < 0; ++q)
      if (legs[q][0] == 0 && legs[(q + L - 1) % L][0] == 1) start = q;
    if (start < 0) return fail(this, 8, "core legs are not in two runs");
  }
  std::vector<int> idx(L);
  for (int i = 0; i < L; ++i) idx[i] = (start + i) % L;
  int n0 = 0;
  if (nc == 2) {
    while (n0 < L && legs[idx[n0]][0] == 0) ++n0;
    for (int i = n0; i < L; ++i)
      if (legs[idx[i]][0] != 1) return fail(this, 8, "core legs are not in two runs");
  } else {
    n0 = L / 2;
  }
  if (n0 < 1 || n0 >= L) return fail(this, 8, "core legs are not in two runs");
  int perm[2][4];
  int cnt[2] = {0, 0};
  for (int i = 0; i < L; ++i) {
    const int k = legs[idx[i]][0];
    if (cnt[k] >= 4) return fail(this, 8, "core leg list too long");
    perm[k][cnt[k]++] = legs[idx[i]][1];
  }
  for (int k = 0; k < nc; ++k) {
    if (nc == 2) perm[k][cnt[k]++] = js[k];
    if (cnt[k] != 4) return fail(this, 8, "core site legs do not match the ring");
    bool seen[4] = {false, false, false, false};
    for (int q = 0; q < 4; ++q) {
      if (perm[k][q] < 0 || perm[k][q] > 3 || seen[perm[k][q]]) return fail(this, 8, "core site legs repeated");
      seen[perm[k][q]] = true;
    }
  }
  // shapes: A (l0, P1, m), B (m, P2, l0), joint J
  const int l0 = ring.sh[idx[0]].l;
  const int m = ring.sh[idx[n0 - 1]].r;
  long long P1 = 1, P2 = 1, capA = 1, capB = 1;
  for (int i = 0; i < n0; ++i) {
    P1 *= ring.sh[idx[i]].p;
    capA = std::max(capA, (long long)l0 * P1 * ring.sh[idx[i]].r);
  }
  for (int i = n0; i < L; ++i) {
    P2 *= ring.sh[idx[i]].p;
    capB = std::max(capB, (long long)m * P2 * ring.sh[idx[i]].r);
  }
  if (ring.sh[idx[L - 1]].r != l0) return fail(this, 8, "the ring does not close");
  const auto& n0d = site_n[rs[0]->gid];
  long long f1 = 1;
  for (int q = 0; q < (nc == 2 ? 3 : 4); ++q) f1 *= (long long)n0d[perm[0][q]] * n0d[perm[0][q]];
  if (f1 != (nc == 2 ? P1 : P1 * P2)) return fail(this, 8, "core site 0 legs disagree with the ring");
  const long long J = nc == 2 ? (long long)n0d[js[0]] * n0d[js[0]] : P2;
  if (nc == 2) {
    const auto& n1d = site_n[rs[1]->gid];
    long long f2 = 1;
    for (int q = 0; q < 3; ++q) f2 *= (long long)n1d[perm[1][q]] * n1d[perm[1][q]];
    if (f2 != P2 || (long long)n1d[js[1]] * n1d[js[1]] != J) return fail(this, 8, "core site 1 legs disagree with the ring");
  }
  const long long LM = (long long)l0 * m;
  const size_t nA = 2 * capA + LM * P1, nB = 2 * capB + LM * P2, nT = P1 * J + P2 * J, nX = 2 * LM * J;
  const int nz = nops + 1;
  DBuf wk, opd;
  if (!wk.ensure(sizeof(C) * (nA + nB + nT + nX + 2 * LM + nz) + 1024, stream)) return fail(this, 2, "allocation failed");
  C* A0 = (C*)wk.p;
  C* A1 = A0 + capA;
  C* Ap = A1 + capA;
  C* B0 = Ap + LM * P1;
  C* B1 = B0 + capB;
  C* Bp = B1 + capB;
  C* T1 = Bp + LM * P2;
  C* T2 = T1 + P1 * J;
  C* X1 = T2 + P2 * J;
  C* X2 = X1 + LM * J;
  C* Dp = X2 + LM * J;                 // per-row dots
  C* ones = Dp + LM;
  C* Zs = ones + LM;
  CK(launch_fill(ones, LM, 1.0, 0.0, stream));
  const size_t op_elems = (size_t)nops * nc * d * d;
  if (nops > 0) {
    if (!opd.ensure(sizeof(double2) * op_elems + 256, stream)) return fail(this, 2, "allocation failed");
    CK(cudaMemcpyAsync(opd.p, ops, sizeof(double2) * op_elems, cudaMemcpyHostToDevice, stream));
  }
  const C one = one_of<C>(), zero = zero_of<C>();
  // product of a run of ring tensors: (l, prod p, r); the rows of each
  // product go in chunks (the GEMM grid's row count is bounded)
  constexpr long long kRows = 1 << 20;
  auto chain = [&](int i0, int i1, C* b0, C* b1) -> const C* {
    const C* cur = ring.t[idx[i0]];
    long long rows = (long long)ring.sh[idx[i0]].l * ring.sh[idx[i0]].p;
    int cols = ring.sh[idx[i0]].r;
    C* out = b0;
    for (int i = i0 + 1; i < i1; ++i) {
      const TShape t = ring.sh[idx[i]];
      for (long long r0 = 0; r0 < rows; r0 += kRows)
        if (launch_zgemm('N', 'N', (int)std::min(kRows, rows - r0), t.p * t.r, cols, one, cur + r0 * cols, cols, 0,
                         ring.t[idx[i]], t.p * t.r, 0, zero, out + r0 * (long long)t.p * t.r, t.p * t.r, 0, 1,
                         stream) != cudaSuccess)
          return nullptr;
      cur = out;
      out = (out == b0) ? b1 : b0;
      rows *= t.p;
      cols = t.r;
    }
    return cur;
  };
  const C* A = chain(0, n0, A0, A1);
  if (!A) return fail(this, 3, "core: ring product failed");
  {
    const int pa[3] = {0, 2, 1};   // (l0, P1, m) -> (l0, m, P1)
    CK(launch_permute3(A, l0, (int)P1, m, pa, Ap, stream));
  }
  {
    const C* B = chain(n0, L, B0, B1);
    if (!B) return fail(this, 3, "core: ring product failed");
    const int pb[3] = {2, 0, 1};   // (m, P2, l0) -> (l0, m, P2)
    CK(launch_permute3(B, m, (int)P2, l0, pb, Bp, stream));
  }
  const double2* tbase = (const double2*)t_dev.p;
  const size_t tsz = (size_t)d * D * D * D * D;
  for (int k = 0; k <= nops; ++k) {          // k = nops: no operator, Z(1)
    const double2* o0 = k < nops ? (const double2*)opd.p + ((size_t)k * nc) * d * d : nullptr;
    CK(launch_fuse(tbase + (size_t)rs[0]->gid * tsz, d, D, n0d.data(), o0, perm[0], T1, stream));
    CK(launch_zgemm('N', 'N', (int)LM, (int)J, (int)P1, one, Ap, (int)P1, 0, T1, (int)J, 0, zero, X1, (int)J, 0, 1,
                    stream));
    const C* Xb = Bp;
    if (nc == 2) {
      const double2* o1 = k < nops ? (const double2*)opd.p + ((size_t)k * nc + 1) * d * d : nullptr;
      CK(launch_fuse(tbase + (size_t)rs[1]->gid * tsz, d, D, site_n[rs[1]->gid].data(), o1, perm[1], T2, stream));
      CK(launch_zgemm('N', 'N', (int)LM, (int)J, (int)P2, one, Bp, (int)P2, 0, T2, (int)J, 0, zero, X2, (int)J, 0, 1,
                      stream));
      Xb = X2;
    }
    // Z = sum_rows sum_j X1[row, j] Xb[row, j]: one CTA per row (batched 1 x 1
    // products), then the sum of the LM row dots
    constexpr long long kBatch = 32768;
    for (long long r0 = 0; r0 < LM; r0 += kBatch)
      CK(launch_zgemm('N', 'T', 1, 1, (int)J, one, X1 + r0 * J, (int)J, J, Xb + r0 * J, (int)J, J, zero, Dp + r0, 1, 1,
                      (int)std::min(kBatch, LM - r0), stream));
    CK(launch_zgemm('N', 'N', 1, 1, (int)LM, one, ones, (int)LM, 0, Dp, 1, 0, zero, Zs + k, 1, 0, 1, stream));
  }
  std::vector<C> hz(nz);
  CK(cudaMemcpyAsync(hz.data(), Zs, sizeof(C) * nz, cudaMemcpyDeviceToHost, stream));
  double ls = 0.0;
  if (int rc = core_ring_result<C>(ring, &ls)) return rc;   // (synchronises)
  const double zr = hz[nops].x, zi = hz[nops].y, den = zr * zr + zi * zi;
  if (!(den > 0.0)) return fail(this, 5, "the core's value vanishes");
  for (int k = 0; k < nops; ++k) {
    const double ar = hz[k].x, ai = hz[k].y;
    re[k] = (ar * zr + ai * zi) / den;
    im[k] = (ai * zr - ar * zi) / den;
  }
  return 0;
}

// ------------------------------------------------------------ ITE (Ch. 3)
//
// One bond update, every step on the device in complex128:
//  * the bond's Edge TN (the pMPS around its two sites) contracted into the
//    dense environment N[K1 K2, B1 B2] (ket legs, bra legs; site 1's three
//    outer legs then site 2's, in ring order);
//  * x = t1, y = t2 as [p, outer legs, bond]; Theta = gate (x y);
//  * the ALS start: the truncated SVD of Theta across the bond, D kept;
//  * ALS half-steps: the normal equations M v_p = c_p of Phi for one tensor
//    with the other fixed (M from N and the fixed tensor, c from N, Theta
//    and the fixed tensor), solved by the least-squares solution from the
//    SVD of M (rcond 1e-13);
//  * Phi = <psi - Theta| N |psi - Theta> after every half-step; the loop
//    stops when a sweep lowers Phi by at most tol Phi_start.

namespace {

StridedView sview(std::initializer_list<long long> dims, std::initializer_list<long long> sstr) {
  StridedView v;
  v.rank = (int)dims.size();
  int q = 0;
  for (long long x : dims) v.dims[q++] = x;
  q = 0;
  for (long long x : sstr) v.sstr[q++] = x;
  long long st = 1;
  for (int k = v.rank - 1; k >= 0; --k) {
    v.dstr[k] = st;
    st *= v.dims[k];
  }
  v.total = st;
  return v;
}

}  // namespace

int Engine::ite_bond(int g1, int k1, const double* gate, int max_sweeps, double tol, std::vector<double>& phi) {
  DeviceScope ds(device);
  phi.clear();
  if (precision != 0) return fail(this, 1, "the ITE update runs in the FP64 mode");
  if (!partitioned || !messages_ready) return fail(this, 8, "partition and messages are required first");
  if (!gate || k1 < 0 || k1 > 3 || max_sweeps < 0) return fail(this, 1, "bad arguments");
  int loc1 = -1;
  const int bid = geom.home_block(g1, &loc1);
  if (bid < 0) return fail(this, 1, "site out of range");
  const Block& blk = geom.blocks[bid];
  const auto& st1 = blk.sites[loc1];
  int t2, i2, j2, k2;
  geom.lat.neighbour(st1[0], st1[1], st1[2], k1, t2, i2, j2, k2);
  const int g2 = geom.lat.site_id(t2, i2, j2);
  if (g2 < 0) return fail(this, 1, "the leg is open");
  auto it2 = std::find(blk.gids.begin(), blk.gids.end(), g2);
  if (it2 == blk.gids.end()) return fail(this, 1, "the ITE update needs both sites of the bond in one block");
  const int loc2 = (int)(it2 - blk.gids.begin());
  const std::vector<int> core = {loc1, loc2};

  CoreRing<double2> ring;
  if (int rc = core_ring<double2>(bid, core, ring)) return rc;
  const Region& R = block_regions[bid];
  const RSite* rs[2] = {nullptr, nullptr};
  for (int q = 0; q < 2; ++q)
    for (const RSite& x : R.sites)
      if (x.inst == 0 && x.local == core[q]) rs[q] = &x;
  if (!rs[0] || !rs[1]) return fail(this, 8, "core site missing from the block region");
  int js[2] = {-1, -1}, njoint = 0;
  for (int s1 = 0; s1 < 4; ++s1)
    for (int s2 = 0; s2 < 4; ++s2)
      if (rs[0]->label[s1] == rs[1]->label[s2]) { js[0] = s1; js[1] = s2; ++njoint; }
  if (njoint != 1 || js[0] != k1) return fail(this, 1, "the two sites must share exactly this one bond");
  const auto& legs = ring.cp.legs;
  const int L = (int)legs.size();
  int start = -1;
  for (int q = 0; q < L && start < 0; ++q)
    if (legs[q][0] == 0 && legs[(q + L - 1) % L][0] == 1) start = q;
  if (start < 0) return fail(this, 8, "core legs are not in two runs");
  std::vector<int> idx(L);
  for (int i = 0; i < L; ++i) idx[i] = (start + i) % L;
  int n0 = 0;
  while (n0 < L && legs[idx[n0]][0] == 0) ++n0;
  int outer[2][3], cnt[2] = {0, 0};
  for (int i = 0; i < L; ++i) {
    const int k = legs[idx[i]][0];
    if ((k == 0) != (i < n0) || cnt[k] >= 3) return fail(this, 8, "core legs are not in two runs");
    outer[k][cnt[k]++] = legs[idx[i]][1];
  }
  if (cnt[0] != 3 || cnt[1] != 3) return fail(this, 8, "a bond core has three outer legs a site");
  const int gid[2] = {rs[0]->gid, rs[1]->gid};
  const auto& na = site_n[gid[0]];
  const auto& nb = site_n[gid[1]];
  long long E1 = 1, E2 = 1;
  for (int q = 0; q < 3; ++q) { E1 *= na[outer[0][q]]; E2 *= nb[outer[1][q]]; }
  const int Db = na[js[0]];
  if (nb[js[1]] != Db) return fail(this, 8, "bond extents differ");
  const long long P1 = E1 * E1, P2 = E2 * E2;
  long long rp1 = 1, rp2 = 1;
  for (int i = 0; i < n0; ++i) rp1 *= ring.sh[idx[i]].p;
  for (int i = n0; i < L; ++i) rp2 *= ring.sh[idx[i]].p;
  if (rp1 != P1 || rp2 != P2) return fail(this, 8, "the Edge TN legs disagree with the sites");
  if (P1 * P2 > (1LL << 26)) return fail(this, 1, "the bond's dense environment is too large (D at most 4)");
  const int l0 = ring.sh[idx[0]].l, m = ring.sh[idx[n0 - 1]].r;
  if (ring.sh[idx[L - 1]].r != l0) return fail(this, 8, "the ring does not close");
  const long long LM = (long long)l0 * m;
  long long capA = 1, capB = 1;
  {
    long long p = 1;
    for (int i = 0; i < n0; ++i) { p *= ring.sh[idx[i]].p; capA = std::max(capA, (long long)l0 * p * ring.sh[idx[i]].r); }
    p = 1;
    for (int i = n0; i < L; ++i) { p *= ring.sh[idx[i]].p; capB = std::max(capB, (long long)m * p * ring.sh[idx[i]].r); }
  }
  const int dd = d;
  const long long dE1 = dd * E1, dE2 = dd * E2, EE = E1 * E2, d2 = (long long)dd * dd;
  const long long n1 = E1 * Db, n2 = E2 * Db, nmax = std::max(n1, n2);
  // scratch layout
  std::vector<std::pair<double2**, long long>> lay;
  double2 *A0, *A1, *Ap, *B0, *B1, *Bp, *Nf, *Nkb, *Nr1, *Nr2, *X, *Y, *XT, *YT, *Gd, *psi1, *psi, *Th, *Thm, *TN, *TNp1,
      *TNp2, *G, *Gr, *MM, *Mt, *cc, *cT, *W, *U, *Rm, *Xd, *Tq;
  lay = {{&A0, capA}, {&A1, capA}, {&Ap, LM * P1}, {&B0, capB}, {&B1, capB}, {&Bp, LM * P2}, {&Nf, P1 * P2},
         {&Nkb, P1 * P2}, {&Nr1, P1 * P2}, {&Nr2, P1 * P2}, {&X, dE1 * Db}, {&Y, dE2 * Db}, {&XT, dE1 * Db},
         {&YT, dE2 * Db}, {&Gd, d2 * d2}, {&psi1, d2 * EE}, {&psi, d2 * EE}, {&Th, d2 * EE}, {&Thm, d2 * EE},
         {&TN, d2 * EE}, {&TNp1, d2 * EE}, {&TNp2, d2 * EE}, {&G, nmax * nmax}, {&Gr, std::max(P1, P2) * Db * Db},
         {&MM, std::max(P1, P2) * Db * Db}, {&Mt, nmax * nmax}, {&cc, nmax * dd}, {&cT, nmax * dd}, {&W, nmax * dd},
         {&U, std::max(nmax * nmax, dE1 * dE2)}, {&Rm, std::max(nmax * nmax, dE1 * dE2)}, {&Xd, d2 * EE},
         {&Tq, d2 * EE}};
  size_t tot = 0;
  for (auto& e : lay) tot += (size_t)((e.second + 31) / 32 * 32);
  DBuf wk, svdw, sc;
  if (!wk.ensure(sizeof(double2) * tot + 256, stream)) return fail(this, 2, "allocation failed");
  {
    size_t off = 0;
    for (auto& e : lay) {
      *e.first = (double2*)wk.p + off;
      off += (size_t)((e.second + 31) / 32 * 32);
    }
  }
  const size_t svd_bytes = std::max(svd_work_bytes((int)nmax, (int)nmax), svd_work_bytes((int)dE1, (int)dE2));
  if (!svdw.ensure(svd_bytes + 256, stream) || !sc.ensure(64, stream)) return fail(this, 2, "allocation failed");
  int* svd_status = (int*)sc.p;
  double* phid = (double*)((char*)sc.p + 16);
  CK(cudaMemsetAsync(svd_status, 0, sizeof(int), stream));
  const double2 one = make_double2(1, 0), zero = make_double2(0, 0);
  constexpr long long kRows = 1 << 20;
  auto chain = [&](int i0, int i1, double2* b0, double2* b1) -> const double2* {
    const double2* cur = ring.t[idx[i0]];
    long long rows = (long long)ring.sh[idx[i0]].l * ring.sh[idx[i0]].p;
    int cols = ring.sh[idx[i0]].r;
    double2* out = b0;
    for (int i = i0 + 1; i < i1; ++i) {
      const TShape t = ring.sh[idx[i]];
      for (long long r0 = 0; r0 < rows; r0 += kRows)
        if (launch_zgemm('N', 'N', (int)std::min(kRows, rows - r0), t.p * t.r, cols, one, cur + r0 * cols, cols, 0,
                         ring.t[idx[i]], t.p * t.r, 0, zero, out + r0 * (long long)t.p * t.r, t.p * t.r, 0, 1,
                         stream) != cudaSuccess)
          return nullptr;
      cur = out;
      out = (out == b0) ? b1 : b0;
      rows *= t.p;
      cols = t.r;
    }
    return cur;
  };
  auto copy = [&](const double2* src, double2* dst, const StridedView& v) { return launch_strided_copy(src, dst, v, stream); };

  // dense environment: N[f1, f2] = sum_{l0, m} A[l0, f1, m] B[m, f2, l0]
  const double2* A = chain(0, n0, A0, A1);
  const double2* B = chain(n0, L, B0, B1);
  if (!A || !B) return fail(this, 3, "ITE: ring product failed");
  {
    const int pa[3] = {1, 2, 0}, pb[3] = {0, 2, 1};
    CK(launch_permute3(A, l0, (int)P1, m, pa, Ap, stream));   // (P1, m, l0)
    CK(launch_permute3(B, m, (int)P2, l0, pb, Bp, stream));   // (m, l0, P2)
  }
  CK(launch_zgemm('N', 'N', (int)P1, (int)P2, (int)LM, one, Ap, (int)LM, 0, Bp, (int)P2, 0, zero, Nf, (int)P2, 0, 1,
                  stream));
  {   // unfuse: (k0 b0 k1 b1 ... k5 b5) -> (k0 .. k5, b0 .. b5)
    long long dims12[12], str12[12];
    for (int q = 0; q < 6; ++q) {
      const int nq = q < 3 ? na[outer[0][q]] : nb[outer[1][q - 3]];
      dims12[2 * q] = dims12[2 * q + 1] = nq;
    }
    long long stv = 1;
    for (int a = 11; a >= 0; --a) { str12[a] = stv; stv *= dims12[a]; }
    StridedView v;
    v.rank = 12;
    for (int q = 0; q < 6; ++q) {
      v.dims[q] = dims12[2 * q];
      v.sstr[q] = str12[2 * q];
      v.dims[6 + q] = dims12[2 * q + 1];
      v.sstr[6 + q] = str12[2 * q + 1];
    }
    long long st = 1;
    for (int k = 11; k >= 0; --k) { v.dstr[k] = st; st *= v.dims[k]; }
    v.total = st;
    CK(copy(Nf, Nkb, v));
  }
  // x, y: [p, outer legs in ring order, bond] gathered from the site tensors
  const long long sz = (long long)dd * D * D * D * D;
  auto sstride = [&](int slot) { long long r = 1; for (int q = slot + 1; q < 4; ++q) r *= D; return r; };
  const double2* tb = (const double2*)t_dev.p;
  CK(copy(tb + gid[0] * sz, X, sview({dd, na[outer[0][0]], na[outer[0][1]], na[outer[0][2]], Db},
                                     {(long long)D * D * D * D, sstride(outer[0][0]), sstride(outer[0][1]),
                                      sstride(outer[0][2]), sstride(js[0])})));
  CK(copy(tb + gid[1] * sz, Y, sview({dd, nb[outer[1][0]], nb[outer[1][1]], nb[outer[1][2]], Db},
                                     {(long long)D * D * D * D, sstride(outer[1][0]), sstride(outer[1][1]),
                                      sstride(outer[1][2]), sstride(js[1])})));
  CK(cudaMemcpyAsync(Gd, gate, sizeof(double2) * d2 * d2, cudaMemcpyHostToDevice, stream));
  // psi = x y over the bond, as [p1 p2, K1 K2]; Theta = gate psi
  auto two_site = [&](const double2* x, const double2* y, double2* out) -> int {
    CK(launch_zgemm('N', 'T', (int)dE1, (int)dE2, Db, one, x, Db, 0, y, Db, 0, zero, psi1, (int)dE2, 0, 1, stream));
    CK(copy(psi1, out, sview({dd, dd, E1, E2}, {E1 * dE2, E2, dE2, 1})));
    return 0;
  };
  if (int rc = two_site(X, Y, psi)) return rc;
  CK(launch_zgemm('N', 'N', (int)d2, (int)EE, (int)d2, one, Gd, (int)d2, 0, psi, (int)EE, 0, zero, Th, (int)EE, 0, 1,
                  stream));
  // TN[p1 p2, B1 B2] = sum_K Theta[p, K] N[K, B]; its two groupings
  CK(launch_zgemm('N', 'N', (int)d2, (int)EE, (int)EE, one, Th, (int)EE, 0, Nkb, (int)EE, 0, zero, TN, (int)EE, 0, 1,
                  stream));
  CK(copy(TN, TNp1, sview({dd, E1, dd, E2}, {dd * EE, E2, EE, 1})));     // [(p1 B1), (p2 B2)]
  CK(copy(TN, TNp2, sview({dd, E2, dd, E1}, {EE, 1, dd * EE, E2})));     // [(p2 B2), (p1 B1)]
  CK(copy(Nkb, Nr1, sview({E1, E1, E2, E2}, {E2 * EE, E2, EE, 1})));    // [K1, B1, K2, B2]
  CK(copy(Nkb, Nr2, sview({E2, E2, E1, E1}, {EE, 1, E2 * EE, E2})));    // [K2, B2, K1, B1]
  // the ALS start: truncated SVD of Theta as [(p1 K1), (p2 K2)]
  CK(copy(Th, Thm, sview({dd, E1, dd, E2}, {dd * EE, E2, EE, 1})));
  CK(launch_svd_trunc(Thm, (int)dE1, (int)dE2, Db, U, Rm, svdw.p, svd_status, stream));
  const int k0 = (int)std::min<long long>(Db, std::min(dE1, dE2));
  CK(cudaMemsetAsync(X, 0, sizeof(double2) * dE1 * Db, stream));
  CK(cudaMemsetAsync(Y, 0, sizeof(double2) * dE2 * Db, stream));
  {
    StridedView v = sview({dE1, k0}, {k0, 1});
    v.dstr[0] = Db;
    v.dstr[1] = 1;
    CK(copy(U, X, v));
    StridedView w = sview({dE2, k0}, {1, dE2});                          // y[(p2 K2), b] = Rem[b, (p2 K2)]
    w.dstr[0] = Db;
    w.dstr[1] = 1;
    CK(copy(Rm, Y, w));
  }
  auto phi_eval = [&](double* out) -> int {
    if (int rc = two_site(X, Y, Xd)) return rc;
    CK(launch_axpy(Th, Xd, d2 * EE, make_double2(-1, 0), stream));
    CK(launch_zgemm('N', 'N', (int)d2, (int)EE, (int)EE, one, Xd, (int)EE, 0, Nkb, (int)EE, 0, zero, Tq, (int)EE, 0,
                    1, stream));
    CK(launch_quad_form(Tq, Xd, d2 * EE, phid, stream));
    CK(cudaMemcpyAsync(out, phid, sizeof(double), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return 0;
  };
  // least-squares solution of M v = c for the d columns of cT: out (n x d)
  auto solve = [&](int n, double2* out) -> int {
    CK(launch_svd_trunc(Mt, n, n, n, U, Rm, svdw.p, svd_status, stream));
    CK(launch_zgemm('C', 'N', n, dd, n, one, U, n, 0, cT, dd, 0, zero, W, dd, 0, 1, stream));
    CK(launch_pinv_rows(W, Rm, n, dd, 1e-13, stream));
    CK(launch_zgemm('C', 'N', n, dd, n, one, Rm, n, 0, W, dd, 0, zero, out, dd, 0, 1, stream));
    return 0;
  };
  // one half-step: the site tensor `var` (outer size Ev) with the other one,
  // `fix` (outer size Ef), fixed
  auto half = [&](bool first) -> int {
    const long long Ev = first ? E1 : E2, Ef = first ? E2 : E1;
    const long long nf = Ef * Db, nv = Ev * Db;
    double2* fix = first ? Y : X;
    double2* var = first ? X : Y;
    // G[(Kf b), (Bf b')] = sum_p conj(fix[p, (Kf b)]) fix[p, (Bf b')]
    CK(launch_zgemm('C', 'N', (int)nf, (int)nf, dd, one, fix, (int)nf, 0, fix, (int)nf, 0, zero, G, (int)nf, 0, 1,
                    stream));
    // Gr[(Kf Bf), (b b')] = G[(Bf b'), (Kf b)]
    CK(copy(G, Gr, sview({Ef, Ef, Db, Db}, {Db, Db * nf, 1, nf})));
    // MM[(Kv Bv), (b b')] = Nr[(Kv Bv), (Kf Bf)] Gr
    CK(launch_zgemm('N', 'N', (int)(Ev * Ev), Db * Db, (int)(Ef * Ef), one, first ? Nr1 : Nr2, (int)(Ef * Ef), 0, Gr,
                    Db * Db, 0, zero, MM, Db * Db, 0, 1, stream));
    // M[(Bv b'), (Kv b)] = MM[Kv, Bv, b, b']
    CK(copy(MM, Mt, sview({Ev, Db, Ev, Db}, {(long long)Db * Db, 1, Ev * Db * Db, Db})));
    // fix^T: [b, (p Kf)]
    CK(copy(fix, first ? YT : XT, sview({Db, dd * Ef}, {1, Db})));
    // c[(p Bv), b'] = TNp[(p Bv), (p' Bf)] conj(fix[(p' Bf), b'])
    CK(launch_zgemm('N', 'C', (int)(dd * Ev), Db, (int)(dd * Ef), one, first ? TNp1 : TNp2, (int)(dd * Ef), 0,
                    first ? YT : XT, (int)(dd * Ef), 0, zero, cc, Db, 0, 1, stream));
    // cT[(Bv b'), p] = c[p, Bv, b']
    CK(copy(cc, cT, sview({Ev, Db, dd}, {Db, 1, Ev * Db})));
    if (int rc = solve((int)nv, cc)) return rc;   // the solution, (Kv b) x p, replaces c
    // var[p, Kv, b] = sol[(Kv b), p]
    CK(copy(cc, var, sview({dd, Ev, Db}, {1, Db * dd, dd})));
    return 0;
  };
  double ph = 0.0;
  if (int rc = phi_eval(&ph)) return rc;
  phi.push_back(ph);
  for (int sw = 0; sw < max_sweeps; ++sw) {
    if (int rc = half(true)) return rc;
    if (int rc = phi_eval(&ph)) return rc;
    phi.push_back(ph);
    if (int rc = half(false)) return rc;
    if (int rc = phi_eval(&ph)) return rc;
    phi.push_back(ph);
    const size_t q = phi.size();
    if (phi[q - 3] - phi[q - 1] <= tol * std::max(std::fabs(phi[0]), 1e-300)) break;
  }
  int hst = 0;
  CK(cudaMemcpyAsync(&hst, svd_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (hst) return fail(this, 5, "an SVD of the ITE update did not converge");
  // the new tensors replace the old ones (open legs at index 0), each / max |entry|
  drop_graphs();
  for (int q = 0; q < 2; ++q) {
    const auto& nn = q == 0 ? na : nb;
    double2* dst = (double2*)t_dev.p + gid[q] * sz;
    CK(cudaMemsetAsync(dst, 0, sizeof(double2) * sz, stream));
    StridedView v = sview({dd, nn[outer[q][0]], nn[outer[q][1]], nn[outer[q][2]], Db}, {0, 0, 0, 0, 0});
    long long st = 1;
    for (int k = 4; k >= 0; --k) { v.sstr[k] = st; st *= v.dims[k]; }
    v.dstr[0] = (long long)D * D * D * D;
    v.dstr[1] = sstride(outer[q][0]);
    v.dstr[2] = sstride(outer[q][1]);
    v.dstr[3] = sstride(outer[q][2]);
    v.dstr[4] = sstride(js[q]);
    CK(copy(q == 0 ? X : Y, dst, v));
    CK(launch_scale_absmax(dst, sz, stream));
  }
  for (auto itf = fused.begin(); itf != fused.end();) {
    if (itf->first.first == gid[0] || itf->first.first == gid[1]) itf = fused.erase(itf);
    else ++itf;
  }
  CK(cudaStreamSynchronize(stream));
  return 0;
}

int Engine::ite(const double* gates, int ndt, const int* bonds, int nbonds, double bp_tol, int bp_iter,
                int als_sweeps, double* energies) {
  if (!gates || ndt < 0 || !bonds || nbonds <= 0 || !energies) return fail(this, 1, "bad arguments");
  const size_t gsz = 2 * (size_t)d * d * d * d;
  std::vector<double> phi;
  for (int k = 0; k < ndt; ++k) {
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q < nbonds; ++q) {
        const int b = pass == 0 ? q : nbonds - 1 - q;
        int its = 0;
        double err = 0.0;
        const int rc = iterate(bp_tol, bp_iter, &its, &err);
        if (rc && rc != 6) return rc;
        if (int rc2 = ite_bond(bonds[2 * b], bonds[2 * b + 1], gates + gsz * k, als_sweeps, 1e-13, phi)) return rc2;
      }
    int its = 0;
    double err = 0.0;
    const int rc = iterate(bp_tol, bp_iter, &its, &err);
    if (rc && rc != 6) return rc;
    if (int rc2 = energy_per_site(&energies[k])) return rc2;
  }
  return 0;
}

}  // namespace bbp
