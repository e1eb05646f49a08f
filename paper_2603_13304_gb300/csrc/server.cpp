// Many BlockBP problems on one GPU: a batched iteration over several
// contexts and a continuous-batching job server.
//
// Every context iterates on its own private root stream (a captured CUDA
// graph per iteration, forked over its worker streams), so the iterations of
// different contexts overlap on the device.  bbp_batch_iterate advances all
// unconverged contexts one synchronous iteration per round.  The server
// admits queued jobs in arrival order while their estimated device footprint
// fits the budget and a slot is free, keeps every admitted job's messages
// resident, relaunches each job as soon as its previous iteration has
// completed (no round barrier), and retires a job when its message error
// reaches its tolerance, its iteration limit is hit, or it fails.  The host
// work of different contexts (context set-up, sweep preparation, graph
// capture, launches) runs on a few host threads at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <exception>
#include <string>
#include <thread>
#include <vector>

#include "../../include/bbp.h"
#include "ctx.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int n_sites_of(int lattice, int Lx, int Ly) { return lattice == BBP_KAGOME ? 3 * Lx * Ly : Lx * Ly; }

// Host threads that prepare and enqueue the iterations of different
// contexts at once: a context's host work (shape simulation, graph capture
// or eager launches) is independent of every other context's.
int host_threads() {
  static const int n = [] {
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(8u, h ? h : 1u));
  }();
  return n;
}

// The workers start on the calling thread's current device (a new host
// thread would otherwise start on device 0).
template <typename F>
void parallel_for(size_t n, F&& f) {
  const int T = (int)std::min<size_t>(n, (size_t)host_threads());
  if (T <= 1) {
    for (size_t i = 0; i < n; ++i) f(i);
    return;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = -1;
  }
  std::atomic<size_t> next{0};
  std::vector<std::thread> ts;
  ts.reserve(T);
  for (int t = 0; t < T; ++t)
    ts.emplace_back([&, dev] {
      if (dev >= 0) cudaSetDevice(dev);
      for (size_t i; (i = next.fetch_add(1)) < n;) f(i);
    });
  for (auto& t : ts) t.join();
}

// ------------------------------------------------ one launch per round
//
// The graph-replayed iterations of a round go to the device as one graph:
// per context the tolerance upload, the context's iteration graph as a child
// node and the download of its convergence word, the contexts independent of
// one another.  Built once per set of (context, capture) ids and relaunched
// while the set repeats (a few sets are kept: the iterations alternate
// between two message parities).
std::atomic<bool> g_single_launch{true};
constexpr size_t kBatchGraphChildren = 128;

struct BatchGraph {
  std::vector<std::pair<unsigned long long, unsigned long long>> key;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_bg_mu;
std::deque<BatchGraph> g_bg;
constexpr size_t kBatchGraphsKept = 32;   // (chunks x two message parities)

int launch_round(bbp_ctx** ctxs, const std::vector<int>& idx, const std::vector<bbp::Engine::Deferred>& ds,
                 cudaStream_t bs) {
  std::vector<std::pair<unsigned long long, unsigned long long>> key(idx.size());
  for (size_t a = 0; a < idx.size(); ++a) key[a] = {ctxs[idx[a]]->eng.uid(), ds[a].uid};
  std::lock_guard<std::mutex> lk(g_bg_mu);
  cudaGraphExec_t exec = nullptr;
  for (auto it = g_bg.begin(); it != g_bg.end(); ++it)
    if (it->key == key) {
      exec = it->exec;
      BatchGraph hit = *it;
      g_bg.erase(it);
      g_bg.push_front(hit);
      break;
    }
  if (!exec) {
    cudaGraph_t G = nullptr;
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return BBP_ERR_CUDA;
    bool ok = true;
    std::map<const void*, cudaGraphNode_t> last;   // contexts of one worker pool run one after another
    for (size_t a = 0; a < ds.size() && ok; ++a) {
      cudaGraphNode_t n1, n2, n3;
      auto it = last.find(ds[a].pool);
      const bool chained = it != last.end();
      cudaGraphNode_t prev = chained ? it->second : nullptr;
      ok = cudaGraphAddMemcpyNode1D(&n1, G, chained ? &prev : nullptr, chained ? 1 : 0, ds[a].tol_dev,
                                    ds[a].host_word, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaGraphAddChildGraphNode(&n2, G, &n1, 1, ds[a].graph) == cudaSuccess &&
           cudaGraphAddMemcpyNode1D(&n3, G, &n2, 1, ds[a].host_word + 1, ds[a].word_dev, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost) == cudaSuccess;
      if (ok) last[ds[a].pool] = n3;
    }
    if (ok) ok = cudaGraphInstantiate(&exec, G, 0) == cudaSuccess;
    cudaGraphDestroy(G);
    if (!ok) {
      cudaGetLastError();
      return BBP_ERR_CUDA;
    }
    if (g_bg.size() >= kBatchGraphsKept) {
      cudaStreamSynchronize(bs);        // (an evicted graph may still run on an earlier round)
      cudaDeviceSynchronize();
      cudaGraphExecDestroy(g_bg.back().exec);
      g_bg.pop_back();
    }
    g_bg.push_front(BatchGraph{key, exec});
  }
  for (int i : idx)
    if (ctxs[i]->eng.defer_before(bs)) return BBP_ERR_CUDA;
  if (cudaGraphLaunch(exec, bs) != cudaSuccess) return BBP_ERR_CUDA;
  for (int i : idx)
    if (ctxs[i]->eng.defer_after(bs)) return BBP_ERR_CUDA;
  return BBP_OK;
}

}  // namespace

// Worker pools shared by groups of contexts: heaviest first, dealt round
// the groups back and forth, so that every group gets a like mix (its arenas
// sized by its heaviest member) and the groups' serial chains balance.
extern "C" bbp_status bbp_share_workers(bbp_ctx** ctxs, int n, int groups) {
  if (!ctxs || n < 0 || groups < 0) return BBP_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return BBP_ERR_ARG;
  try {
    if (groups == 0) {
      for (int i = 0; i < n; ++i)
        if (ctxs[i]->eng.use_workers(nullptr)) return BBP_ERR_CUDA;
      return BBP_OK;
    }
    std::vector<std::pair<double, int>> w(n);
    for (int i = 0; i < n; ++i) {
      const bbp::Engine& e = ctxs[i]->eng;
      const double D2 = (double)e.D * e.D;
      w[i] = {(double)e.geom.lat.n_sites() * (double)e.chi * e.chi * D2 * std::max(D2, (double)e.chi), i};
    }
    std::sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<std::shared_ptr<bbp::WorkerPool>> pools(std::min(groups, std::max(n, 1)));
    for (auto& p : pools) p = std::make_shared<bbp::WorkerPool>();
    const int G = (int)pools.size();
    for (int r = 0; r < n; ++r) {
      const int lap = r / G, pos = r % G;
      const int g = (lap & 1) ? G - 1 - pos : pos;
      if (ctxs[w[r].second]->eng.use_workers(pools[g])) return BBP_ERR_CUDA;
    }
    return BBP_OK;
  } catch (const std::bad_alloc&) {
    return BBP_ERR_OOM;
  } catch (...) {
    return BBP_ERR_CUDA;
  }
}

extern "C" bbp_status bbp_batch_single_launch(int on) {
  g_single_launch.store(on != 0);
  return BBP_OK;
}

extern "C" bbp_status bbp_batch_iterate(bbp_ctx** ctxs, int n, double tol, int max_iter, int* iters_out,
                                        double* err_out, int* status_out) {
  if (!ctxs || n < 0 || !iters_out || !err_out || !status_out || max_iter < 0 || !(tol >= 0.0))
    return BBP_ERR_ARG;
  try {
    std::vector<int> active;
    for (int i = 0; i < n; ++i) {
      iters_out[i] = 0;
      err_out[i] = INFINITY;
      status_out[i] = BBP_OK;
      if (!ctxs[i]) {
        status_out[i] = BBP_ERR_ARG;
        continue;
      }
      const int rc = ctxs[i]->eng.iter_begin();
      if (rc) status_out[i] = rc;
      else active.push_back(i);
    }
    const bool single = g_single_launch.load() && active.size() > 1;
    std::vector<cudaStream_t> chunk_streams;
    for (int round = 0; round < max_iter && !active.empty(); ++round) {
      std::vector<int> rcs(active.size(), 0);
      parallel_for(active.size(), [&](size_t a) {
        try {
          ctxs[active[a]]->eng.iter_tol = tol;
          ctxs[active[a]]->eng.defer_graph = single;
          rcs[a] = ctxs[active[a]]->eng.iter_launch();
          ctxs[active[a]]->eng.defer_graph = false;
        } catch (...) {
          rcs[a] = BBP_ERR_CUDA;
        }
      });
      std::vector<int> launched, deferred;
      std::vector<bbp::Engine::Deferred> ds;
      for (size_t a = 0; a < active.size(); ++a) {
        if (rcs[a]) {
          status_out[active[a]] = rcs[a];
          continue;
        }
        launched.push_back(active[a]);
        bbp::Engine::Deferred d;
        if (ctxs[active[a]]->eng.deferred(d)) {
          deferred.push_back(active[a]);
          ds.push_back(d);
        }
      }
      // the round's graph in chunks of whole worker pools, about
      // kBatchGraphChildren contexts each, every chunk on its own stream
      // (the contexts of one pool stay in one chunk, in launch order)
      if (!deferred.empty()) {
        std::vector<size_t> ord(deferred.size());
        for (size_t a = 0; a < ord.size(); ++a) ord[a] = a;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return ds[x].pool < ds[y].pool; });
        size_t chunk = 0;
        for (size_t a0 = 0; a0 < ord.size(); ++chunk) {
          size_t a1 = a0;
          while (a1 < ord.size() && (a1 - a0 < kBatchGraphChildren || ds[ord[a1]].pool == ds[ord[a1 - 1]].pool)) ++a1;
          std::vector<int> ci;
          std::vector<bbp::Engine::Deferred> cd;
          for (size_t a = a0; a < a1; ++a) {
            ci.push_back(deferred[ord[a]]);
            cd.push_back(ds[ord[a]]);
          }
          while (chunk_streams.size() <= chunk) {
            cudaStream_t cs = nullptr;
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BBP_ERR_CUDA;
            chunk_streams.push_back(cs);
          }
          if (launch_round(ctxs, ci, cd, chunk_streams[chunk]) != BBP_OK) {
            for (int i : ci) ctxs[i]->eng.defer_after(chunk_streams[chunk]);   // (finish reports the failed round)
            for (int i : ci) status_out[i] = BBP_ERR_CUDA;
          }
          a0 = a1;
        }
      }
      std::vector<int> next;
      for (int i : launched) {
        double e = INFINITY;
        const bool failed = status_out[i] != BBP_OK;   // (its round's launch failed)
        const int rc = ctxs[i]->eng.iter_finish(&e);
        ++iters_out[i];
        err_out[i] = e;
        if (rc) status_out[i] = rc;
        else if (!failed && !(e <= tol)) next.push_back(i);
      }
      active.swap(next);
    }
    for (cudaStream_t cs : chunk_streams) cudaStreamDestroy(cs);   // (their work completes first)
    for (int i = 0; i < n; ++i) {
      if (!ctxs[i]) continue;
      ctxs[i]->eng.iter_end();
      if (status_out[i] == BBP_OK && !(err_out[i] <= tol)) status_out[i] = BBP_NOT_CONVERGED;
    }
    bbp_status worst = BBP_OK;
    for (int i = 0; i < n; ++i)
      if (status_out[i] != BBP_OK && (worst == BBP_OK || worst == BBP_NOT_CONVERGED)) worst = (bbp_status)status_out[i];
    return worst;
  } catch (const std::bad_alloc&) {
    return BBP_ERR_OOM;
  } catch (...) {
    return BBP_ERR_CUDA;
  }
}

// ------------------------------------------------------------------ server

struct bbp_server {
  struct Job {
    long long id = 0;
    bbp_job spec{};
    std::vector<double> tensors, edges;
    size_t bytes = 0;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    bbp_ctx* ctx = nullptr;
    int iters = 0;
    double err = INFINITY;
    int status = BBP_OK;
    bool in_flight = false;
  };
  size_t budget = 0;
  int max_active = 1;
  size_t used = 0;
  long long next_id = 1;
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::vector<Job*> finished;   // completed, not yet taken

  ~bbp_server() {
    for (Job* j : queue) delete j;
    for (Job* j : active) drop(j);
    for (Job* j : finished) drop(j);
  }
  void drop(Job* j) {
    if (j->ctx) bbp_destroy(j->ctx);
    delete j;
  }
};

namespace {

// Device bytes a job holds while resident: site tensors, fused tensors and
// messages of its context plus the workspace of each of its worker streams.
size_t job_bytes(const bbp_job& j, int streams) {
  const size_t z = j.precision == BBP_FP64 ? 16 : 8;
  const size_t ns = (size_t)n_sites_of(j.lattice, j.Lx, j.Ly);
  const size_t D2 = (size_t)j.D * j.D, chi = (size_t)j.chi;
  const size_t blk = (size_t)j.bx * j.by * (j.lattice == BBP_KAGOME ? 3 : 1);
  const size_t nblocks = blk ? (ns + blk - 1) / blk : 0;
  const size_t k = j.lattice == BBP_KAGOME ? 2 * (size_t)j.bx : (size_t)std::max(j.bx, j.by);
  const size_t msgs = nblocks * 4 * 2 * k * chi * chi * D2 * z;
  const size_t tens = ns * (size_t)j.d * D2 * D2 * 16;
  const size_t fused = ns * 4 * D2 * D2 * D2 * D2 * z;
  const size_t seg = chi * chi * D2 * std::max(D2, chi) * z;
  return msgs + tens + fused + (size_t)streams * 16 * seg + (64u << 20);
}

int start_job(bbp_server::Job* j) {
  // the context's caller stream is the legacy one: its iterations run on
  // the context's own non-blocking streams, so jobs do not serialise on it
  const bbp_job& s = j->spec;
  bbp_status rc = bbp_create_peps(&j->ctx, s.lattice, s.Lx, s.Ly, s.periodic, s.d, s.D, j->tensors.data(), 0, nullptr);
  if (rc) return rc;
  if ((rc = bbp_partition_blocks(j->ctx, s.bx, s.by))) return rc;
  if ((rc = bbp_set_options(j->ctx, s.chi, s.precision, 1.0, 0))) return rc;
  if ((rc = bbp_set_execution(j->ctx, 1, s.streams > 0 ? s.streams : 4))) return rc;
  if (s.precision != BBP_FP64 && (rc = bbp_set_power_iters(j->ctx, s.power_iters >= 0 ? s.power_iters : 1))) return rc;
  if ((rc = bbp_init_messages(j->ctx, j->edges.data()))) return rc;
  const int e = j->ctx->eng.iter_begin();
  return e;
}

}  // namespace

extern "C" bbp_status bbp_server_create(bbp_server** out, size_t hbm_budget_bytes, int max_active) {
  if (!out || max_active < 1 || hbm_budget_bytes == 0) return BBP_ERR_ARG;
  try {
    bbp_server* s = new bbp_server();
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    *out = s;
    return BBP_OK;
  } catch (...) {
    return BBP_ERR_OOM;
  }
}

extern "C" void bbp_server_destroy(bbp_server* s) {
  if (!s) return;
  try {
    delete s;
  } catch (...) {
  }
}

extern "C" size_t bbp_job_footprint_bytes(const bbp_job* job) {
  if (!job) return 0;
  return job_bytes(*job, job->streams > 0 ? job->streams : 4);
}

extern "C" bbp_status bbp_server_submit(bbp_server* s, const bbp_job* job, long long* id_out) {
  if (!s || !job || !id_out || !job->host_tensors || !job->edge_mats) return BBP_ERR_ARG;
  if (job->tensor_dtype != 0 && job->tensor_dtype != 1) return BBP_ERR_ARG;
  if (job->Lx < 1 || job->Ly < 1 || job->d < 1 || job->D < 1 || job->chi < 1 || job->max_iter < 0 || !(job->tol >= 0.0))
    return BBP_ERR_ARG;
  try {
    auto* j = new bbp_server::Job();
    j->id = s->next_id++;
    j->spec = *job;
    const size_t ns = (size_t)n_sites_of(job->lattice, job->Lx, job->Ly);
    const size_t D4 = (size_t)job->D * job->D * job->D * job->D;
    const size_t nt = 2 * ns * job->d * D4;
    if (job->tensor_dtype == 1) {
      const float* f = (const float*)job->host_tensors;
      j->tensors.assign(f, f + nt);
    } else {
      const double* t = (const double*)job->host_tensors;
      j->tensors.assign(t, t + nt);
    }
    j->edges.assign(job->edge_mats, job->edge_mats + 2 * ns * 4 * job->D * job->D);
    j->spec.host_tensors = nullptr;
    j->spec.edge_mats = nullptr;
    j->bytes = job_bytes(*job, job->streams > 0 ? job->streams : 4);
    j->t_submit = now_s();
    s->queue.push_back(j);
    *id_out = j->id;
    return BBP_OK;
  } catch (...) {
    return BBP_ERR_OOM;
  }
}

// One scheduling step: admit what fits, launch an iteration of every
// admitted job that has none in flight, wait (up to timeout_ms) until at
// least one in-flight iteration completes, then finish every completed one
// and retire the jobs that are done.
extern "C" bbp_status bbp_server_step(bbp_server* s, double timeout_ms, int* n_queued, int* n_active, int* n_finished) {
  if (!s) return BBP_ERR_ARG;
  try {
    // admission: arrival order, footprint within budget, free slot
    std::vector<bbp_server::Job*> admitted;
    while (!s->queue.empty() && (int)(s->active.size() + admitted.size()) < s->max_active) {
      bbp_server::Job* j = s->queue.front();
      if (s->used + j->bytes > s->budget && !(s->active.empty() && admitted.empty())) break;
      s->queue.pop_front();
      s->used += j->bytes;
      j->t_start = now_s();
      admitted.push_back(j);
    }
    std::vector<int> rcs(admitted.size(), 0);
    parallel_for(admitted.size(), [&](size_t a) {
      try {
        rcs[a] = start_job(admitted[a]);
      } catch (...) {
        rcs[a] = BBP_ERR_CUDA;
      }
    });
    for (size_t a = 0; a < admitted.size(); ++a) {
      bbp_server::Job* j = admitted[a];
      if (rcs[a]) {
        j->status = rcs[a];
        j->t_done = now_s();
        s->finished.push_back(j);
      } else {
        s->active.push_back(j);
      }
    }
    std::vector<bbp_server::Job*> idle;
    for (bbp_server::Job* j : s->active)
      if (!j->in_flight && j->status == BBP_OK) idle.push_back(j);
    parallel_for(idle.size(), [&](size_t a) {
      bbp_server::Job* j = idle[a];
      int rc;
      try {
        j->ctx->eng.iter_tol = j->spec.tol;
        rc = j->ctx->eng.iter_launch();
      } catch (...) {
        rc = BBP_ERR_CUDA;
      }
      if (rc) j->status = rc;
      else j->in_flight = true;
    });
    const double t0 = now_s();
    std::vector<bbp_server::Job*> keep;
    for (; !s->active.empty();) {
      bool any = false;
      for (bbp_server::Job* j : s->active)
        if (!j->in_flight || j->ctx->eng.iter_ready()) any = true;
      if (any || (now_s() - t0) * 1e3 > timeout_ms) break;
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (bbp_server::Job* j : s->active) {
      if (j->in_flight && j->ctx->eng.iter_ready()) {
        double e = INFINITY;
        const int rc = j->ctx->eng.iter_finish(&e);
        j->in_flight = false;
        ++j->iters;
        j->err = e;
        if (rc) j->status = rc;
      }
      const bool done = j->status != BBP_OK || (!j->in_flight && (j->err <= j->spec.tol || j->iters >= j->spec.max_iter));
      if (done && !j->in_flight) {
        j->ctx->eng.iter_end();
        if (j->status == BBP_OK && !(j->err <= j->spec.tol)) j->status = BBP_NOT_CONVERGED;
        j->t_done = now_s();
        s->finished.push_back(j);
      } else {
        keep.push_back(j);
      }
    }
    s->active.swap(keep);
    if (n_queued) *n_queued = (int)s->queue.size();
    if (n_active) *n_active = (int)s->active.size();
    if (n_finished) *n_finished = (int)s->finished.size();
    return BBP_OK;
  } catch (const std::bad_alloc&) {
    return BBP_ERR_OOM;
  } catch (...) {
    return BBP_ERR_CUDA;
  }
}

// Completed jobs not yet taken: id, status, iterations, final error, time in
// queue and total latency (submit to completion), in seconds.
extern "C" bbp_status bbp_server_poll(bbp_server* s, long long* ids, int* status, int* iters, double* err,
                                      double* wait_s, double* latency_s, int cap, int* n_out) {
  if (!s || !n_out || cap < 0) return BBP_ERR_ARG;
  int n = 0;
  for (bbp_server::Job* j : s->finished) {
    if (n >= cap) break;
    if (ids) ids[n] = j->id;
    if (status) status[n] = j->status;
    if (iters) iters[n] = j->iters;
    if (err) err[n] = j->err;
    if (wait_s) wait_s[n] = j->t_start - j->t_submit;
    if (latency_s) latency_s[n] = j->t_done - j->t_submit;
    ++n;
  }
  *n_out = n;
  return BBP_OK;
}

// Hand a completed job's context to the caller (who then owns and destroys
// it) or, with ctx_out NULL, release it.  Its footprint leaves the budget.
extern "C" bbp_status bbp_server_take(bbp_server* s, long long id, bbp_ctx** ctx_out) {
  if (!s) return BBP_ERR_ARG;
  for (size_t i = 0; i < s->finished.size(); ++i) {
    bbp_server::Job* j = s->finished[i];
    if (j->id != id) continue;
    s->finished.erase(s->finished.begin() + (long)i);
    s->used -= std::min(s->used, j->bytes);
    if (ctx_out) {
      *ctx_out = j->ctx;
      j->ctx = nullptr;   // the caller owns it now
    }
    s->drop(j);
    return BBP_OK;
  }
  return BBP_ERR_ARG;
}
