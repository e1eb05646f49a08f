// BlockBP engine: device state, sweep executor, iteration and observables.
//
// One implementation serves both precisions: the sweep executor, the
// iteration driver and the observables are templates on the element type
// (double2 = complex128 FP64 path, float2 = complex64 mixed path) and are
// dispatched on `precision`.  Device buffers are untyped; message tensors,
// fused tensors and sweep workspaces hold elements of the current precision.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <memory>
#include <mutex>
#include <map>
#include <string>
#include <vector>

#include "geom.h"
#include "plan.h"

namespace bbp {

// ------------------------------------------------------------- allocation

void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
void set_allocator(void* (*a)(size_t, void*, void*), void (*f)(void*, void*, void*), void* user);

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  bool ensure(size_t n, cudaStream_t st);   // grow-only; false on OOM
  void release();
  ~DBuf() { release(); }
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
};

// ---------------------------------------------------------------- messages

struct Message {
  bool open = false;                   // open boundary: fixed trivial message (all dims 1)
  std::vector<int> Dleg;               // bond dimension of each fused leg
  std::vector<TShape> sh[2];           // shapes of the two buffers
  DBuf buf[2];
  DBuf lrn;                            // learning step / Hermitisation: k sum tensors of 4 cap, k of cap
  size_t cap = 0;                      // elements per tensor
  int cur = 0;
  template <typename C> C* tensor(int which, int q) const { return (C*)buf[which].p + (size_t)q * cap; }
  int k() const { return (int)Dleg.size(); }
};

// ------------------------------------------------------------ sweep work

struct SweepWork {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  DBuf arena;
  size_t elem = 0, cap_t = 0, cap_seg = 0, cap_x = 0, svd_bytes = 0, nslots = 0, cap_d = 0, tc_bytes = 0;
  unsigned long long gen = 0;          // advances with every new layout of the arena
  std::vector<void*> slot;
  void *S[2] = {nullptr, nullptr}, *R[2] = {nullptr, nullptr};
  void *qrA = nullptr, *qrQ = nullptr, *qrR = nullptr, *tau = nullptr, *X = nullptr;
  void* svd = nullptr;
  void* tc = nullptr;                  // tensor-core absorb scratch (packed operands, FP32 product)
  double* logscale = nullptr;
  int* status = nullptr;               // [0] SVD sweep limit, [1] tensor-core pipeline timeout
  double2* scal = nullptr;             // scalar outputs (mps_dot)
  void** ptrs = nullptr;               // device pointer tables (K4, dot)
  int* ints = nullptr;                 // device shape tables
  double2* k4 = nullptr;               // K4 scratch (complex128)
  double2 *dX0 = nullptr, *dX1 = nullptr, *dQ = nullptr, *dR = nullptr, *dtau = nullptr;   // distance (complex128)
  bool reserve(size_t elem, size_t cap_t, size_t cap_seg, size_t cap_x, size_t svd_bytes, size_t nslots, size_t cap_d,
               size_t tc_bytes);
};

// The worker streams and workspace arenas of one or more contexts.  Contexts
// that share a pool (bbp_share_workers) run their iterations one after
// another: every use locks the pool on the host, waits for last_done and
// records it again when its work is enqueued.
class Engine;
struct WorkerPool {
  std::vector<SweepWork*> w;
  cudaEvent_t last_done = nullptr;
  std::mutex mu;
  std::vector<Engine*> pending;        // members whose deferred graph (bound to the arenas) awaits its launch
  WorkerPool();
  ~WorkerPool();
  WorkerPool(const WorkerPool&) = delete;
  WorkerPool& operator=(const WorkerPool&) = delete;
};

struct SweepJob {
  const SweepPlan* plan = nullptr;
  ShapeTrace tr;
  std::vector<const void*> node_tensor;      // site: fused T permuted (in..., out...); message: raw (l, p, r)
  std::vector<std::array<int, 5>> node_fuse; // site fused on the fly (node_tensor null): gid, perm[4]
  std::vector<TShape> node_shape;            // message nodes: tensor shape
  std::vector<const void*> start;            // start chain tensors, canonical orientation
  std::vector<TShape> start_shape;           // their shapes (canonical orientation)
  std::vector<void*> dest;                   // final MPS tensors, canonical order
};

using OpList = std::vector<std::pair<std::array<int, 2>, const double*>>;   // (instance, local) -> device d x d c128

template <typename C> struct CoreRing;   // the pMPS of one core on the device (engine.cpp)

class Engine {
 public:
  Geometry geom;
  int d = 2, D = 2, chi = 8, precision = 0, power_iters = 1, power_iters64 = 6;
  double alpha = 1.0;                  // learning step: alpha new + (1 - alpha) old (Sec. 2.3.3)
  bool hermitise = false;              // replace each new message by its Hermitian part
  bool learning() const { return alpha != 1.0 || hermitise; }
  int tc_mode = 0;                     // absorb contraction: 0 SIMT GEMM, 1 tcgen05 TF32 split, 2 tcgen05 BF16 split
  bool use_graphs = true;              // replay a captured CUDA graph per iteration
  int max_streams = 16;                // sweep jobs run on up to this many streams
  size_t fuse_cache_max = size_t(2) << 30;   // fused site tensors kept when they take at most this; else fused per use
  cudaStream_t stream = nullptr;
  int device = -1;                     // device current at create(); every iteration call runs on it
  bool partitioned = false;
  std::string last_error;

  DBuf t_dev;                                   // site tensors [n][d][D]^4, complex128
  std::vector<std::array<int, 4>> site_n;       // used extent per leg (1 open, D)
  std::map<std::pair<int, int>, DBuf> fused;    // (gid, perm code) -> fused tensor (current precision)
  std::map<std::pair<int, int>, Message> msgs;  // incoming message per (block, face)
  std::map<std::pair<int, int>, SweepPlan> plans;   // (block, face) -> plan (single-block regions)
  std::vector<Region> block_regions;                // single-block region per block
  std::shared_ptr<WorkerPool> workers;
  DBuf dist_dev, op_dev;
  long long launches_per_iter = 0;
  double flops_per_iter = 0.0;
  bool messages_ready = false;
  int n_iterations = 0;

  ~Engine();
  size_t elem() const { return precision == 0 ? sizeof(double2) : sizeof(float2); }
  bool fuse_on_the_fly() const;
  int create(int lattice, int Lx, int Ly, int periodic, int d, int D, const double* host_t, cudaStream_t s);
  int partition(int bx, int by);
  int set_precision(int p);
  int init_messages(const double* edge_mats);
  int iterate(double tol, int max_iter, int* iters, double* err);
  // split iteration (several contexts in flight): begin, then launch/finish
  // pairs, then end; see engine.cpp
  int iter_begin();
  int iter_launch();
  int iter_finish(double* err);
  int iter_end();
  bool iter_ready() const { return root_out && cudaEventQuery(root_out) == cudaSuccess; }
  int contract_batch(const std::vector<std::vector<std::array<int, 2>>>& coords, const std::vector<OpList>& ops,
                     std::vector<double>& logscale, std::vector<double>& re, std::vector<double>& im);
  int bond_region(int g1, int k1, std::vector<std::array<int, 2>>& coords, std::array<int, 2>& key1,
                  std::array<int, 2>& key2);
  int energy_per_site(double* e);
  int bond_energies(const std::vector<std::array<int, 2>>& bonds, std::vector<double>& out);
  int log_norm(double* out);
  int get_message(int block, int face, int* k, int* shapes, double* data, size_t cap);
  // Core extraction (Sec. 2.3, "Core"): two bubbles from the bottom and top
  // faces of `block` that leave the sites `core` (local indices) open, joined
  // by the zipper into a periodic MPS around the core.  Output on the host,
  // complex128: the pMPS tensors in cyclic order (shapes l, p, r), the
  // (position in `core`, slot) of each tensor's physical leg, and the log of
  // the scale factored out of the two bubbles.
  int core_pmps(int block, const std::vector<int>& core, std::vector<TShape>& shapes,
                std::vector<std::array<int, 2>>& legs, std::vector<double2>& data, double* logscale);
  // Local quantities of a core of one site, or of the two ends of a bond
  // (the Edge TN): for each of nops operator sets (ncore host d x d
  // complex128 operators each, set k site q at ops + 2 d d (k ncore + q)),
  // <O_k> = Z(O_k) / Z(1), the core contracted exactly with its pMPS.
  int core_expect(int block, const std::vector<int>& core, const double* ops, int nops, double* re, double* im);
  // ITE update of one bond (Ch. 3, "ITE update step"; FP64 mode, both ends in
  // one block): the bond leaving site g1 through slot k1 takes the two-site
  // gate (host d^2 x d^2 complex128 over (s1 s2)), then ALS on the bond's
  // Edge TN brings it back to bond D; the new site tensors replace the old
  // ones, each divided by its largest entry.  phi: Phi after the SVD start
  // and after every ALS half-step.
  int ite_bond(int g1, int k1, const double* gate, int max_sweeps, double tol, std::vector<double>& phi);
  // Full ITE (Alg. 2): for each of ndt gates, every bond of the list, then
  // the list backwards, is updated after BlockBP runs to bp_tol; energies
  // receives the energy per site after each gate's pass.
  int ite(const double* gates, int ndt, const int* bonds, int nbonds, double bp_tol, int bp_iter, int als_sweeps,
          double* energies);

 private:
  SweepWork* work(size_t i);
  template <typename C> const C* fused_tensor(int gid, const int perm[4]);
  template <typename C> int init_messages_t(const double* edge_mats);
  template <typename C>
  int fill_job(const Region& R, const SweepPlan& plan, SweepJob& job, const OpList& ops, std::vector<DBuf*>& tmp);
  int reserve_workers(const std::vector<SweepJob>& jobs, int nstreams);
  template <typename C> int run_sweep(SweepJob& job, SweepWork& w);
  template <typename C>
  int finalize_message(Message& m, int which, SweepWork& w, cudaStream_t s, double* dist_slot, bool with_distance);
  template <typename C> int compress_lrn(Message& m, std::vector<TShape>& sh, SweepWork& w, cudaStream_t s);
  template <typename C> int learn_message(Message& m, int which, SweepWork& w, cudaStream_t s);
  int reserve_learning(Message& m);
  template <typename C> int iter_launch_t();
  template <typename C>
  int contract_batch_t(const std::vector<std::vector<std::array<int, 2>>>& coords, const std::vector<OpList>& ops,
                       std::vector<double>& logscale, std::vector<double>& re, std::vector<double>& im);
  template <typename C> int log_norm_t(double* out);
  template <typename C> int get_message_t(int block, int face, int* k, int* shapes, double* data, size_t cap);
  template <typename C>
  int core_pmps_t(int block, const std::vector<int>& core, std::vector<TShape>& shapes,
                  std::vector<std::array<int, 2>>& legs, std::vector<double2>& data, double* logscale);
  template <typename C> int core_ring(int block, const std::vector<int>& core, CoreRing<C>& ring);
  template <typename C> int core_ring_result(CoreRing<C>& ring, double* logscale);
  template <typename C>
  int core_expect_t(int block, const std::vector<int>& core, const double* ops, int nops, double* re, double* im);
  void job_needs(const SweepJob& job, size_t need[7]) const;
  // one captured iteration per message-buffer parity, valid while the
  // signature (shapes and device pointers of every job) is unchanged
  struct IterGraph {
    unsigned long long sig = 0;
    unsigned long long in_sig = 0;     // inputs only: message shapes and buffers, workspaces
    cudaGraph_t graph = nullptr;       // the captured graph (a child of a batch's graph)
    cudaGraphExec_t exec = nullptr;    // instantiated on the first launch of its own
    unsigned long long uid = 0;        // unique over the process, per capture
    long long launches = 0;
    double flops = 0.0;
    std::vector<std::vector<TShape>> out_shapes;   // per update: the outgoing message's shapes
  };
  unsigned long long input_signature(int nstreams) const;
  IterGraph graphs[2];
  unsigned long long last_in_sig[2] = {0, 0};   // inputs of the last iteration of each parity
  cudaStream_t root = nullptr;         // private root of every iteration (and of its capture)
  cudaEvent_t root_in = nullptr, root_in2 = nullptr, root_out = nullptr;
  double* h_word = nullptr;            // pinned: [0] tol of the iteration, [1] largest change, [2] flags (int)

 public:
  double iter_tol = 0.0;               // tolerance the device compares the iteration's largest change with
  bool last_converged = false;         // converged bit of the last finished iteration's word

 private:
  bool in_flight = false;
  bool pending_launch = false;         // the iteration in flight waits for the caller's batch launch
  cudaEvent_t root_pre = nullptr;      // the root's work before a deferred launch
  unsigned long long uid_ = 0;
  bool launched_graph = false;         // the iteration in flight is a graph replay
  int launched_parity = 0;
  long long graph_tag(int parity) const { return (long long)(((uintptr_t)this >> 4) * 2 + (uintptr_t)parity); }

 public:
  void drop_graphs();
  // Deferred graph launch (bbp_batch_iterate): with defer_graph set, an
  // iteration that would replay or newly capture its graph leaves the launch
  // (the tolerance upload, the graph, the word download) to the caller, who
  // puts it into one graph over many contexts; deferred() describes it.
  bool defer_graph = false;
  struct Deferred {
    cudaGraph_t graph = nullptr;
    unsigned long long uid = 0;
    double* tol_dev = nullptr;         // <- host_word[0], 8 bytes, before the graph
    double* word_dev = nullptr;        // -> host_word + 1, 16 bytes, after it
    double* host_word = nullptr;
    const void* pool = nullptr;        // contexts of one worker pool run in launch order
  };
  bool deferred(Deferred& d) const;
  // orders the batch stream after this context's root stream, and the root
  // (and the iteration's completion event) after the batch's launch
  int defer_before(cudaStream_t batch);
  int defer_after(cudaStream_t batch);
  // launches a deferred iteration on this context's own root stream now
  // (the pool's lock held by the caller)
  int launch_deferred_now();
  unsigned long long uid() const { return uid_; }
  // join a worker pool (null: a private one again); waits for this
  // context's work in flight
  int use_workers(std::shared_ptr<WorkerPool> p);
  WorkerPool& pool_ref();

 private:
  unsigned long long iter_signature(const std::vector<SweepJob>& jobs, int nstreams) const;
  long long sweep_launches = 0;
  double sweep_flops = 0.0;
};

int fail(Engine* e, int status, const std::string& msg);

}  // namespace bbp
