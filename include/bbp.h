/*
 * bbp.h -- C ABI of the GB300 BlockBP message-update engine.
 *
 * The engine approximately contracts the double-layer network <psi|psi> of a
 * PEPS by Block Belief Propagation (arxiv 2603.13304, Ch. 2): the lattice is
 * cut into blocks; each block sends to every neighbouring block an MPS
 * "message" obtained by contracting the block with all its other incoming
 * messages (Eq. of the BlockBP update, Sec. 2.2) by a boundary-MPS sweep with
 * truncation bond dimension chi (Sec. 1.1.3); all messages are updated
 * synchronously until they stop changing (Alg. 1).  Local expectation values
 * follow from a block contracted with its converged incoming messages.
 *
 * Conventions
 *  - Complex numbers are interleaved (re, im) IEEE doubles ("complex128").
 *  - Every function returns a bbp_status; on failure bbp_last_error(ctx)
 *    (or bbp_last_error(NULL) for failures without a context) describes it.
 *    Nothing is thrown across the ABI.
 *  - Host buffers are owned by the caller and never retained after a call.
 *    Device memory is owned by the context; it is taken from the allocator
 *    installed with bbp_set_allocator (default cudaMalloc / cudaFree).
 *  - All device work is ordered on the CUDA stream given at creation; calls
 *    that return host values synchronise that stream.
 *  - A context is not thread-safe; distinct contexts are independent.
 *
 * Input layout of PEPS tensors ("site tensors"): complex128
 * [n_sites][d][D][D][D][D], the four virtual legs in slot order:
 *   square  (Lx x Ly sites): site r*Lx + c (row r from the top, column c);
 *           slots (up, right, down, left).  On an open boundary the outward
 *           leg is closed with the unit vector e_0 (only index 0 is read).
 *   Kagome  (Lx x Ly unit cells, always periodic): unit cell u = j*Lx + i
 *           holds sites 3u (A), 3u+1 (B = A + a1/2), 3u+2 (C = A + a2/2);
 *           slots A: B(i,j), C(i,j), B(i-1,j), C(i,j-1)
 *                 B: A(i,j), C(i,j), A(i+1,j), C(i+1,j-1)
 *                 C: A(i,j), B(i,j), A(i,j+1), B(i-1,j+1).
 * A fused (double-layer) leg index is ket * D + bra.
 */
#ifndef BBP_H
#define BBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bbp_ctx bbp_ctx;

typedef enum {
  BBP_OK = 0,
  BBP_ERR_ARG = 1,          /* invalid argument or size                         */
  BBP_ERR_OOM = 2,          /* device allocation failed                          */
  BBP_ERR_CUDA = 3,         /* a CUDA call failed                                */
  BBP_ERR_TILING = 4,       /* the block partition breaks the rules of Sec. 2.2.2 */
  BBP_ERR_NUMERIC = 5,      /* NaN/Inf or an SVD that did not converge           */
  BBP_NOT_CONVERGED = 6,    /* max_iter reached; messages remain valid           */
  BBP_ERR_TIMEOUT = 7,      /* a bounded device wait ran out                     */
  BBP_ERR_STATE = 8         /* call out of order (e.g. iterate before partition) */
} bbp_status;

typedef enum { BBP_SQUARE = 0, BBP_KAGOME = 1 } bbp_lattice;
typedef enum { BBP_FP64 = 0, BBP_TF32 = 1, BBP_BF16 = 2, BBP_FP32 = 3 } bbp_precision;
typedef enum { BBP_BOTTOM = 0, BBP_RIGHT = 1, BBP_TOP = 2, BBP_LEFT = 3 } bbp_face;

/* Device allocator used by every context created afterwards.  alloc returns
 * NULL on failure; free releases a pointer returned by alloc.  user is passed
 * back verbatim.  Passing NULL functions restores cudaMalloc / cudaFree. */
typedef void* (*bbp_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*bbp_free_fn)(void* ptr, void* stream, void* user);
void bbp_set_allocator(bbp_alloc_fn alloc, bbp_free_fn free_fn, void* user);

/* Create a PEPS context (Sec. 1.1.2, PEPS; Sec. 2.1, double layer).
 * lattice: BBP_SQUARE (periodic 0 = open, 1 = torus) or BBP_KAGOME
 * (periodic must be 1).  d: physical dimension; D: bond dimension (<= 8).
 * host_tensors: layout above, d * D^4 entries per site, interleaved
 * (re, im): dtype 0 = complex128 (doubles), 1 = complex64 (floats); copied
 * to the device (complex64 entries are widened to complex128 there, where
 * the fusion reads them).  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream). */
bbp_status bbp_create_peps(bbp_ctx** out, int lattice, int Lx, int Ly, int periodic, int d, int D,
                           const void* host_tensors, int dtype, void* cuda_stream);

/* Cut the lattice into blocks (Sec. 2.2.2): square blocks of bx x by sites;
 * Kagome L x L parallelograms of unit cells with bx = by = L >= 2
 * (N_T = 3 L^2, Sec. 2.3.1).  Fails with BBP_ERR_TILING when a block would
 * not tile the lattice or a bond would leave a face diagonally. */
bbp_status bbp_partition_blocks(bbp_ctx* ctx, int bx, int by);

/* chi: truncation bond dimension of the boundary MPS (Sec. 1.1.3), 1..64.
 * precision: BBP_FP64 -- every tensor complex128 (the reference path,
 *   agrees with the FP64 oracle to 1e-10); each truncation of a large split
 *   Z runs a subspace iteration with b = 2 chi directions (six power steps by
 *   default, bbp_set_power_iters) that reaches the exact truncation to
 *   rounding, finished by a complex128 one-sided Jacobi of the b x b factor;
 *   small splits take the exact Jacobi directly.
 * BBP_FP32 -- tensors and contractions complex64; each truncation reduces a
 *   large matrix Z to b = chi + max(8, chi/2) directions by a randomised
 *   subspace iteration (bbp_set_power_iters steps, default 1; Householder
 *   orthonormalisation), runs a complex64 one-sided Jacobi on the b x b
 *   factor and finishes it in complex128 (the pairs across the chi cut are
 *   rotated again in double; singular values and their selection in double);
 *   message norms, phases, distances and log-scales stay double.
 * BBP_TF32 / BBP_BF16 -- as BBP_FP32, with the absorb contraction (the
 *   dense X^T S product of each swallow) and the segment merges on the
 *   tensor cores: operands split into high and low TF32 (or BF16) parts,
 *   hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM (tcgen05).
 *   A pipeline wait that times out makes bbp_iterate return BBP_ERR_TIMEOUT.
 * alpha: learning step (Sec. 2.3.3, Eq. of the learning step), 0 <= alpha
 *   <= 1: the message that replaces the old one is alpha new + (1 - alpha)
 *   old, the MPS sum compressed back to bond chi (left-canonical QR sweep,
 *   then truncated SVDs from the right) and normalised; 1 = plain update.
 * Must be called before bbp_init_messages.  seed is reserved. */
bbp_status bbp_set_options(bbp_ctx* ctx, int chi, int precision, double alpha, uint64_t seed);

/* Hermitisation of messages (Sec. 2.3.3, "Hermitize MPSs"): on = 1 replaces
 * every new message by its Hermitian part (M + M^dagger) / 2 as an operator
 * on the fused (ket, bra) legs, compressed to bond chi as for the learning
 * step and normalised; applied before the learning step.  Default 0. */
bbp_status bbp_set_hermitise(bbp_ctx* ctx, int on);

/* Randomised truncation (no counterpart in the thesis, whose truncation is
 * an exact SVD): number of subspace-iteration power steps before the reduced
 * SVD, 0..8, for the precision already set by bbp_set_options: complex64
 * modes (default 1, b = chi + max(8, chi/2) directions) or BBP_FP64
 * (default 6, b = 2 chi directions, which reaches the exact truncation to
 * rounding on the BlockBP splits; smaller matrices always take the exact
 * one-sided Jacobi).  Fewer steps are faster and less accurate when the
 * spectrum decays slowly. */
bbp_status bbp_set_power_iters(bbp_ctx* ctx, int power_iters);

/* Execution options (no counterpart in the thesis; they change how the same
 * arithmetic is scheduled, not what it computes).  use_graphs = 1 (default)
 * captures one synchronous iteration, every sweep of it forked over up to
 * max_streams CUDA streams (1..64, default 16), into a CUDA graph and
 * replays it while shapes and buffers stay the same; 0 launches eagerly. */
bbp_status bbp_set_execution(bbp_ctx* ctx, int use_graphs, int max_streams);

/* The fused double-layer site tensors (K1, D^8 entries each, one per site
 * and sweep direction) are kept on the device while they take at most
 * max_bytes together (default 2 GiB); above it every site is fused into the
 * sweep's scratch right before its absorb, each iteration, and nothing is
 * kept.  Results are the same either way. */
bbp_status bbp_set_fuse_cache(bbp_ctx* ctx, size_t max_bytes);

/* Initial messages (Alg. 1, "random MPS"): every incoming message becomes a
 * bond-1 MPS whose leg j carries the D x D matrix edge_mats[s][k] of the
 * receiving site s and its slot k.  edge_mats: complex128 [n_sites][4][D][D].
 * Messages are normalised to unit norm with <I|M> real positive. */
bbp_status bbp_init_messages(bbp_ctx* ctx, const double* edge_mats);

/* Synchronous BlockBP iterations (Alg. 1, Eq. of the BlockBP update) until the
 * largest message change ||M_new - M_old|| (unit-norm, phase-fixed messages)
 * is <= tol, or max_iter iterations.  iters_out / err_out (may be NULL)
 * receive the iterations done and the last largest change.  Returns
 * BBP_NOT_CONVERGED when max_iter was reached (messages stay valid). */
bbp_status bbp_iterate(bbp_ctx* ctx, double tol, int max_iter, int* iters_out, double* err_out);

/* <O> for a one- or two-site operator with the converged messages.
 * ns = 1: op is d x d complex128 on site sites[0], inserted as a whole.
 * ns = 2: op is (d*d) x (d*d) complex128 on the pair (sites[0], its
 *   neighbour through slot sites[1]), basis index s0 * d + s1; it is
 *   expanded in the product basis |a0><b0| (x) |a1><b1|, one contraction per
 *   nonzero entry.  If the two sites lie in different blocks the union of
 *   both blocks is contracted.
 * The block (or union) is contracted with all its incoming messages by a
 * sweep to its top face; <O> = Z(O) / Z(1).  A truncated sweep is not linear
 * in the inserted operator, so the expansion above is part of the result. */
bbp_status bbp_expect_local(bbp_ctx* ctx, const double* op, int ns, const int* sites, double* re_out,
                            double* im_out);

/* Reduced density matrix of nsites (1 or 2) sites of one block: rdm_out
 * receives (d^n x d^n) complex128, trace 1, basis index s0 * d + s1.
 * For nsites = 2 the sites may be any two sites of that block. */
bbp_status bbp_block_rdm(bbp_ctx* ctx, int block, const int* sites, int nsites, double* rdm_out);

/* <O1 (x) O2> on the bond that leaves site `site` through leg slot `slot`
 * (Sec. 4.2 observables; reading E for bonds across blocks): O1 acts on
 * `site`, O2 on its neighbour; both host d x d complex128 operators are
 * inserted whole in one contraction (the scheme of bbp_energy_per_site, whose
 * bond terms are the three products S^a (x) S^a).  Results in re_out, im_out. */
bbp_status bbp_expect_product(bbp_ctx* ctx, const double* op1, const double* op2, int site, int slot, double* re_out,
                              double* im_out);

/* Heisenberg bond energies <S_i . S_j> (Sec. 4.2), d = 2: for nbonds bonds
 * given as (site, slot) pairs in site_slots, each the sum of three product
 * insertions S^a (x) S^a as in bbp_energy_per_site; all contractions run as
 * one batch.  e_out: host array of nbonds doubles. */
bbp_status bbp_bond_energies(bbp_ctx* ctx, const int* site_slots, int nbonds, double* e_out);

/* Heisenberg energy per site, sum over all nearest-neighbour bonds of
 * <S_i . S_j> (Eq. of the AFM Heisenberg Hamiltonian, Sec. 4.2) divided by the
 * number of sites; d must be 2. */
bbp_status bbp_energy_per_site(bbp_ctx* ctx, double* e_out);

/* Bethe-form log-norm: sum_a log Z_a - sum_pairs log <M_a->b, M_b->a>
 * (real part), Z_a = block a with all incoming messages. */
bbp_status bbp_norm(bbp_ctx* ctx, double* log_norm_out);

/* Copy the incoming message of (block, face) to the host.  k_out receives
 * the number of tensors, shapes_out (capacity 3*64 ints) the (l, p, r) of each,
 * data_out (capacity cap doubles) the tensors back to back, row-major. */
bbp_status bbp_get_message(bbp_ctx* ctx, int block, int face, int* k_out, int* shapes_out, double* data_out,
                           size_t cap);

/* Core extraction (Sec. 2.3, "Core"): with the current messages, two
 * boundary-MPS sweeps start from the bottom and top faces of `block`,
 * truncate to chi like the message update, and leave the core sites open;
 * the bottom bubble swallows every node before the core's last site in the
 * bottom-up order, the top bubble every node after it.  They meet at two
 * front lines, which the zipper contracts exactly, leaving a periodic MPS
 * (pMPS) around the core, one tensor per open leg of the core.
 * core_sites: ncore distinct global site ids of `block`.  Outputs, in
 * caller-owned host buffers:
 *   len_out       L, the number of pMPS tensors (at most cap_len);
 *   shapes_out    3 L ints, (l, p, r) of each tensor in cyclic order; the r
 *                 of tensor L-1 equals the l of tensor 0;
 *   legs_out      2 L ints, (position in core_sites, leg slot 0..3) of the
 *                 core leg that each tensor's index p joins;
 *   data_out      the tensors back to back, row-major (l, p, r), complex128
 *                 interleaved, at most cap doubles;
 *   logscale_out  natural log of the scale the two bubbles factored out.
 * The core's value with operators inserted is the exact contraction of its
 * fused tensors with the pMPS.  Errors: BBP_ERR_ARG (block or site out of
 * range, a core whose open legs do not face both bubbles, buffers too
 * small), BBP_ERR_STATE (no partition or messages), BBP_ERR_NUMERIC (an
 * SVD of a bubble reached its sweep limit). */
bbp_status bbp_core_pmps(bbp_ctx* ctx, int block, const int* core_sites, int ncore, int cap_len, int* len_out,
                         int* shapes_out, int* legs_out, double* data_out, size_t cap, double* logscale_out);

/* Local quantities of a core (Sec. 2.3, "Core", "Edge"): the core is one
 * site, or the two ends of a bond (its pMPS is then the bond's Edge TN).
 * The core's fused tensors, with operators inserted, are contracted exactly
 * with the pMPS of bbp_core_pmps on the device: <O_k> = Z(O_k) / Z(1).
 * core_sites: ncore (1 or 2) global site ids of `block`; for 2 they must
 * share exactly one bond.  ops: nops sets of ncore host d x d complex128
 * operators O[s, s'] (interleaved), set k site q at ops + 2 d d (k ncore + q).
 * re_out, im_out: nops doubles each.  Errors as bbp_core_pmps;
 * BBP_ERR_NUMERIC also when Z(1) vanishes. */
bbp_status bbp_core_expect(bbp_ctx* ctx, int block, const int* core_sites, int ncore, const double* ops, int nops,
                           double* re_out, double* im_out);

/* ITE update of one bond (Ch. 3, "ITE update step"), FP64 mode, both sites
 * in one block, D at most 4: the bond leaving `site` through leg `slot`
 * takes the two-site gate (host d^2 x d^2 complex128 over (s_site,
 * s_neighbour), e.g. exp(-dt h)); then, with the bond's Edge TN from the
 * current messages as the environment N, alternating least squares brings
 * the bond back to D: from the truncated SVD of the evolved pair, each
 * half-step minimises Phi = <psi - psi'| N |psi - psi'> over one tensor with
 * the other fixed (least squares, rcond 1e-13), until a sweep lowers Phi by
 * at most tol Phi_start or max_sweeps sweeps ran.  The two new tensors
 * replace the old ones, each divided by its largest entry; the messages are
 * kept.  phi_out (capacity phi_cap) receives Phi after the start and after
 * every half-step, n_phi_out their number. */
bbp_status bbp_ite_bond(bbp_ctx* ctx, int site, int slot, const double* gate, int max_sweeps, double tol,
                        double* phi_out, int phi_cap, int* n_phi_out);

/* Full ITE (Alg. 2): for each of ndt gates (host, d^2 x d^2 complex128 each,
 * e.g. exp(-dt h / 2)), the nbonds bonds (site, slot pairs), then the same
 * bonds backwards (second-order splitting), each updated as bbp_ite_bond
 * (at most als_sweeps sweeps) after BlockBP runs to bp_tol (at most
 * bp_max_iter iterations, from the current messages); energies_out (ndt
 * doubles) receives the Heisenberg energy per site after each gate's pass. */
bbp_status bbp_ite(bbp_ctx* ctx, const double* gates, int ndt, const int* bonds, int nbonds, double bp_tol,
                   int bp_max_iter, int als_sweeps, double* energies_out);

/* Device bytes the context would hold for the given problem (estimate). */
size_t bbp_footprint_bytes(int lattice, int n_sites, int D, int chi, int bx, int by, int precision);

/* Number of blocks and of message updates per iteration. */
bbp_status bbp_info(bbp_ctx* ctx, int* n_blocks, int* n_updates, int* n_sites);

/* Statistics of the last bbp_iterate call: kernel launches per iteration and
 * the algorithmic flops of one iteration, counted as 8 l P Q r real flops for
 * every absorb contraction (one complex multiply-add = 8 flops; l, r the
 * outer bonds of the merged segment, P, Q the in- and out-leg products);
 * factorisations are not counted. */
bbp_status bbp_stats(bbp_ctx* ctx, long long* launches_per_iter, double* flops_per_iter);

const char* bbp_last_error(const bbp_ctx* ctx);
void bbp_destroy(bbp_ctx* ctx);

/* ---------------------------------------------------------------------
 * Many problems on one GPU (no counterpart in the thesis).
 * ------------------------------------------------------------------- */

/* Iterate n contexts together: each round launches one synchronous
 * iteration of every context that has not converged and then reads all
 * their errors; a context leaves when its error <= tol or it fails.  The
 * contexts whose iteration replays a captured graph (all of them once their
 * bond dimensions have settled) go to the device as one graph launch per
 * round for every 128 or so of them (whole worker pools per graph, each
 * graph on its own stream), every context's iteration graph a child node
 * (independent, so they overlap on the device); the others launch eagerly
 * on their own streams.  Per context: iterations done, final error and status
 * (BBP_NOT_CONVERGED after max_iter rounds).  Returns BBP_OK,
 * BBP_NOT_CONVERGED, or the first failure among the contexts.
 * bbp_batch_single_launch(0) launches every context's graph separately
 * instead (the default is 1). */
bbp_status bbp_batch_single_launch(int on);
/* Worker streams and workspace arenas shared by groups of contexts: the n
 * contexts are dealt into `groups` pools (heaviest first, back and forth, so
 * that the groups get like mixes); the contexts of one pool run their
 * iterations one after another (in a batch round, in the order of ctxs) and
 * the pool's arenas are sized by its largest member, so that many contexts
 * fit the device.  groups = 0 gives every context a private pool again.
 * Waits for the contexts' work in flight. */
bbp_status bbp_share_workers(bbp_ctx** ctxs, int n, int groups);
bbp_status bbp_batch_iterate(bbp_ctx** ctxs, int n, double tol, int max_iter, int* iters_out, double* err_out,
                             int* status_out);

/* A BlockBP job for the server: the arguments of bbp_create_peps,
 * bbp_partition_blocks, bbp_set_options and bbp_init_messages, the stopping
 * rule (tol, max_iter), the worker streams of its context (<= 0: 4) and the
 * power steps of the complex64 truncation (< 0: 1).  Host arrays are copied
 * by bbp_server_submit. */
typedef struct {
  int lattice, Lx, Ly, periodic, d, D, bx, by, chi, precision;
  double tol;
  int max_iter, streams, power_iters;
  const void* host_tensors;   /* [n_sites][d][D]^4, complex128 or complex64 (tensor_dtype) */
  const double* edge_mats;    /* complex128 [n_sites][4][D][D] */
  int tensor_dtype;           /* 0 = complex128, 1 = complex64, as for bbp_create_peps */
} bbp_job;

typedef struct bbp_server bbp_server;

/* Continuous batching: queued jobs are admitted in arrival order while the
 * sum of the admitted jobs' footprints (bbp_job_footprint_bytes) stays
 * within hbm_budget_bytes and fewer than max_active are resident; admitted
 * jobs keep their messages on the device and each is relaunched as soon as
 * its previous iteration completes; a job finishes at error <= tol, at
 * max_iter iterations or on failure.  One thread drives a server. */
bbp_status bbp_server_create(bbp_server** out, size_t hbm_budget_bytes, int max_active);
size_t bbp_job_footprint_bytes(const bbp_job* job);
bbp_status bbp_server_submit(bbp_server* s, const bbp_job* job, long long* id_out);
/* Admit, launch, wait up to timeout_ms for an iteration to complete, finish
 * and retire; reports the queue, resident and finished counts. */
bbp_status bbp_server_step(bbp_server* s, double timeout_ms, int* n_queued, int* n_active, int* n_finished);
/* Finished jobs not yet taken (up to cap): id, status, iterations, final
 * error, seconds queued and seconds from submit to completion. */
bbp_status bbp_server_poll(bbp_server* s, long long* ids, int* status, int* iters, double* err, double* wait_s,
                           double* latency_s, int cap, int* n_out);
/* Remove a finished job; with ctx_out its context passes to the caller (who
 * destroys it with bbp_destroy), otherwise it is destroyed. */
bbp_status bbp_server_take(bbp_server* s, long long id, bbp_ctx** ctx_out);
void bbp_server_destroy(bbp_server* s);

/* Live kernel timing (no counterpart in the thesis): select one kernel class
 * (0 off, 1 one-sided Jacobi, 2 randomised-range orthonormalisation,
 * 3 Householder QR, 4 tensor-core GEMM, 5 SIMT absorb GEMM, 6 every SIMT
 * complex GEMM); every later
 * launch of it, eager or inside a captured iteration, is bracketed by CUDA
 * events on its own stream.  bbp_iterate adds the completed launches;
 * bbp_ktimer_read returns launches, total milliseconds and algorithmic flops
 * since the last read (and resets them).  Selecting clears all records;
 * select before the iterations whose graphs should carry the events. */
void bbp_ktimer_select(int kernel_class);
bbp_status bbp_ktimer_read(long long* launches, double* ms, double* flops);

/* ---------------------------------------------------------------------
 * Kernel-level entry points (device pointers, for unit tests and tools).
 * All take a cudaStream_t and return after enqueueing the work.
 * ------------------------------------------------------------------- */

/* K1, double-layer fusion (Sec. 2.1): t: device [d][D]^4; n[4]: used extent
 * per leg (1 or D); perm[4]: output axis q is source leg perm[q]; op: device
 * d x d or NULL; T: device output with prod n[perm[q]]^2 entries. */
bbp_status bbp_k_fuse(const double* t, int d, int D, const int* n, const double* op, const int* perm, double* T,
                      void* stream);

/* K3, truncated SVD (Sec. 1.1.1): Z (m x n, device, row-major) = U S V^H;
 * keep k = min(chi, m, n) largest; writes U (m x k) and Rem = S V^H (k x n).
 * work: device scratch of bbp_k_svd_work_bytes(m, n) bytes; status: device
 * int, set to 1 if the sweep limit was reached (never cleared: zero it first). */
size_t bbp_k_svd_work_bytes(int m, int n);
bbp_status bbp_k_svd_trunc(const double* Z, int m, int n, int chi, double* U, double* Rem, void* work, int* status,
                           void* stream);

/* Allocation-free variant of bbp_k_svd_trunc (the thesis has no counterpart;
 * this serves callers that cannot allocate device memory when they need the
 * SVD: real-time loops that must not enter the allocator, since cudaMalloc
 * can synchronise the device, and hosts whose device memory is owned by
 * another runtime with a budget fixed at start-up).
 * Same inputs, outputs and status as bbp_k_svd_trunc, without `work`: the
 * scratch is a fixed device array of 8 MiB + 64 KiB that every GPU loading
 * the library holds until exit, enough for bbp_k_svd_work_bytes(m, n) up to
 * that size (e.g. 512 x 512).  Larger sizes return BBP_ERR_ARG.  It calls no
 * allocator.  The first call on a device loads the array there (CUDA loads
 * modules lazily) and looks up its device address (with that device
 * current); make that first call before any stream capture.  All calls on a
 * device share the array: calls that overlap on the same GPU race. */
bbp_status bbp_k_svd_trunc_noalloc(const double* Z, int m, int n, int chi, double* U, double* Rem, int* status,
                                   void* stream);

/* Work counters of the last bbp_k_svd_trunc that used `work`: Jacobi sweeps
 * and rotations applied (synchronises the stream).  Feeds the flop model. */
bbp_status bbp_k_svd_stats(const void* work, int m, int n, int* sweeps, long long* rotations, void* stream);

/* Householder QR (Sec. 2.3.3 canonical moves): A (m x n, device, destroyed)
 * = Q (m x k) R (k x n), k = min(m, n); tau: device scratch of k complex. */
bbp_status bbp_k_qr(double* A, int m, int n, double* Q, double* R, double* tau, void* stream);

/* Householder QR of tall panels (Sec. 2.3.3 canonical moves; the range
 * orthonormalisation of the truncation) on a cluster of up to 16 CTAs, each
 * holding a row slice in shared memory.  A: device, batch panels of m x n
 * (m >= n, row-major, not modified) at a stride of m * n elements; Q (m x n
 * per panel, may equal A) and R (n x n per panel, upper triangular with a
 * real diagonal) are written when not NULL.  c64 = 1: complex64 entries,
 * 0: complex128.  cluster: CTAs per panel, 0 = automatic; otherwise at
 * least bbp_k_panel_cluster(c64, m, n) (the fewest whose shared memory holds
 * the panel with Q; 0 when even 16 do not) and at most 16.  A call with
 * Q = NULL needs a little less shared memory (no reflector scalars), so it
 * may fit where bbp_k_panel_cluster reports 0.  Each CTA caches 32, 64, ...
 * rows per warp lane (complex64 up to 256 rows a CTA, complex128 up to 128),
 * and a CTA beyond the rows a given cluster needs holds none.  BBP_ERR_ARG
 * when m < n or the panel does not fit. */
int bbp_k_panel_cluster(int c64, int m, int n);
bbp_status bbp_k_panel_qr(int c64, const void* A, int m, int n, void* Q, void* R, int batch, int cluster,
                          void* stream);

/* The engine's truncated SVD (Sec. 1.1.1) with the randomised range
 * reduction (see bbp_set_power_iters): Z (m x n, device, row-major) -> U
 * (m x k) and Rem = S V^H (k x n), k = min(chi, m, n), chi <= 64.
 * c64 = 1: complex64 entries; a subspace iteration with b = chi +
 * max(8, chi/2) directions whose b x b reduced factor is finished in
 * complex128.  c64 = 0: complex128 entries, b = 2 chi directions, the
 * reduced factor by complex128 Jacobi.  Matrices too small to gain from the
 * reduction take the exact one-sided Jacobi.  power_iters: 0..8.
 * tensor_cores = 1 (complex64 only): the range-finder products run as
 * split-TF32 tcgen05 GEMMs (device int err, set to 1 on a pipeline timeout,
 * as for bbp_k_tc_gemm); 0: SIMT GEMMs (err may be NULL).  work: device
 * scratch of bbp_k_svd_work_bytes_rand(c64, m, n, chi, tensor_cores) bytes;
 * status as for bbp_k_svd_trunc. */
size_t bbp_k_svd_work_bytes_rand(int c64, int m, int n, int chi, int tensor_cores);
bbp_status bbp_k_svd_trunc_rand(int c64, const void* Z, int m, int n, int chi, void* U, void* Rem, void* work,
                                int* status, int power_iters, int tensor_cores, int* err, void* stream);

/* K2 on the tensor cores (tcgen05.mma, TMEM accumulator, TMA-fed operands).
 * Real GEMM C (M x N, device fp32, row stride ldc) = alpha * A * B with
 * A row-major M x K (row stride lda) and B given transposed, Bt row-major
 * N x K (row stride ldb).  bf16 = 0: TF32 operands stored as fp32;
 * bf16 = 1: BF16 operands.  A and Bt must be 16-byte aligned and lda, ldb
 * multiples of 16 bytes; ragged M, N, K are zero-filled by TMA.  err: device
 * int set to 1 when a pipeline wait timed out (never cleared). */
bbp_status bbp_k_tc_gemm(int bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C, long long ldc,
                         int M, int N, int K, float alpha, int* err, void* stream);
/* The same GEMM with an explicit tile: bn (output columns of a CTA: 64,
 * 128 or 256) and group_m >= 1 (M tiles that sweep the N tiles together).
 * bbp_k_tc_gemm takes the autotuner's tile for its shape, else the size rule
 * (bn 128 above N = 64, else 64; group_m 16). */
bbp_status bbp_k_tc_gemm_tile(int bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C,
                              long long ldc, int M, int N, int K, float alpha, int bn, int group_m, int* err,
                              void* stream);

/* Tile autotuner of the tensor-core GEMM (process-wide; thread-safe).
 * bbp_autotune_record(1) collects the shape (precision, M, N, K) of every
 * later tensor-core GEMM launch that has no table entry, for example during
 * an eager first iteration; bbp_autotune_run times every candidate tile of
 * each collected shape on scratch operands it allocates (synchronously, on
 * its own stream; not inside a graph capture), keeps the fastest, sets
 * *n_tuned, and writes the whole table to cache_path when it is not NULL
 * (one line "tc bf16 M N K bn group_m microseconds" per shape).
 * bbp_autotune_load merges a table written that way (*n_loaded entries).
 * Every table change advances a generation that the contexts' captured
 * iteration graphs check, so later iterations re-capture with the new tiles.
 * Tiles change only the order of the work, never the arithmetic of an
 * output element. */
bbp_status bbp_autotune_record(int on);
bbp_status bbp_autotune_run(const char* cache_path, int* n_tuned);
bbp_status bbp_autotune_load(const char* cache_path, int* n_loaded);
bbp_status bbp_autotune_info(int* n_entries, int* n_pending, unsigned long long* generation);
bbp_status bbp_autotune_clear(void);

/* The absorb contraction of Sec. 2.3.3 on the tensor cores:
 * R[a] (Q x r) = X^T (Q x P) S[a] (P x r) for a < l, complex, row-major,
 * X: P x Q, S: l x P x r, R: l x Q x r; c64 = 1 for complex64 data, 0 for
 * complex128.  Both operands are scaled by a power of two and split into
 * high and low parts in the operand type (bf16 = 0: TF32, 1: BF16); the three
 * products hi*hi + hi*lo + lo*hi accumulate in FP32 in one real GEMM.  work:
 * device scratch of bbp_k_tc_absorb_bytes(...) bytes; err as above. */
size_t bbp_k_tc_absorb_bytes(int bf16, int P, int Q, int l, int r);
bbp_status bbp_k_tc_absorb(int bf16, int c64, const void* X, int P, int Q, const void* S, int l, int r, void* R,
                           void* work, int* err, void* stream);

/* ALU throughput microbenchmark (no counterpart in the thesis; it measures
 * the FP64 and FP32 denominators of the roofline fractions): blocks x 256
 * threads run iters rounds of 8 independent FMA chains in FP64 (fp64 = 1) or
 * FP32.  out: device scratch of 8 bytes (written only to keep the chains
 * live).  Returns after enqueueing; *flops_out receives the flop count of the
 * launch, so the caller's event timing gives the rate. */
bbp_status bbp_k_fma_peak(int fp64, int blocks, int iters, void* out, double* flops_out, void* stream);

/* Host-side plan of one boundary-MPS sweep (no GPU needed): for block `block`
 * and out face `face`, the swallow order as (kind, id) pairs: kind 0 = site
 * (id = global site id), kind 1 = message tensor (id = face * 1024 + index),
 * and per step the number of in- and out-legs.  out: capacity cap ints,
 * 4 ints per step: kind, id, nin, nout.  n_steps_out receives the count. */
bbp_status bbp_plan_debug(int lattice, int Lx, int Ly, int periodic, int bx, int by, int block, int face, int* out,
                          int cap, int* n_steps_out);

/* Host-side plan of a core extraction (no GPU needed; see bbp_core_pmps):
 * for the core sites core_sites (global ids) of `block`, steps_out receives
 * the swallow order of the bottom bubble and then of the top bubble, 4 ints
 * per step as in bbp_plan_debug (capacity cap ints); info_out 7 ints: steps
 * of the bottom bubble, steps of the top bubble, boundary lengths n and m of
 * the two bubbles, the shared end runs a and c of the zipper, and the number
 * L of pMPS tensors; legs_out 2 L ints (capacity 2 * cap_len): the (position
 * in core_sites, slot) of each pMPS tensor's physical leg. */
bbp_status bbp_core_plan_debug(int lattice, int Lx, int Ly, int periodic, int bx, int by, int block,
                               const int* core_sites, int ncore, int* steps_out, int cap, int* info_out, int* legs_out,
                               int cap_len);

#ifdef __cplusplus
}
#endif

#endif /* BBP_H */
