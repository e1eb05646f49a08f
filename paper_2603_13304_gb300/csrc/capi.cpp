// extern "C" boundary of the BlockBP engine (contract in include/bbp.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/bbp.h"
#include "ctx.h"
#include "engine.h"
#include "kernels.h"


namespace {
thread_local std::string g_err;

bbp_status set_err(bbp_status s, const std::string& m) {
  g_err = m;
  return s;
}

bbp_status from(bbp_ctx* c, int rc) {
  if (rc != 0) g_err = c->eng.last_error;
  return (bbp_status)rc;
}

bbp_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BBP_OK;
  return set_err(BBP_ERR_CUDA, cudaGetErrorString(e));
}

template <typename F>
bbp_status guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return set_err(BBP_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_err(BBP_ERR_STATE, e.what());
  } catch (...) {
    return set_err(BBP_ERR_STATE, "unknown exception");
  }
}
}  // namespace

extern "C" {

void bbp_set_allocator(bbp_alloc_fn alloc, bbp_free_fn free_fn, void* user) {
  if (!alloc || !free_fn) bbp::set_allocator(nullptr, nullptr, nullptr);
  else bbp::set_allocator(alloc, free_fn, user);
}

bbp_status bbp_create_peps(bbp_ctx** out, int lattice, int Lx, int Ly, int periodic, int d, int D,
                           const void* host_tensors, int dtype, void* cuda_stream) {
  return guarded([&]() -> bbp_status {
    if (!out) return set_err(BBP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (dtype != 0 && dtype != 1) return set_err(BBP_ERR_ARG, "dtype must be 0 (complex128) or 1 (complex64)");
    if (!host_tensors) return set_err(BBP_ERR_ARG, "host_tensors is NULL");
    std::vector<double> wide;
    const double* t = (const double*)host_tensors;
    if (dtype == 1) {
      if (d < 1 || d > 4 || D < 1 || D > 8 || Lx <= 0 || Ly <= 0 || Lx > 4096 || Ly > 4096)
        return set_err(BBP_ERR_ARG, "d must be 1..4, D 1..8, and the lattice size in range");
      const size_t ns = (size_t)(lattice == BBP_KAGOME ? 3 : 1) * Lx * Ly;
      const size_t n = 2 * ns * d * D * D * D * D;
      const float* f = (const float*)host_tensors;
      wide.assign(f, f + n);
      t = wide.data();
    }
    bbp_ctx* c = new bbp_ctx();
    int rc = c->eng.create(lattice, Lx, Ly, periodic, d, D, t, (cudaStream_t)cuda_stream);
    if (rc) {
      g_err = c->eng.last_error;
      delete c;
      return (bbp_status)rc;
    }
    *out = c;
    return BBP_OK;
  });
}

bbp_status bbp_partition_blocks(bbp_ctx* ctx, int bx, int by) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  return guarded([&] { return from(ctx, ctx->eng.partition(bx, by)); });
}

bbp_status bbp_set_options(bbp_ctx* ctx, int chi, int precision, double alpha, uint64_t seed) {
  (void)seed;
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (chi < 1 || chi > 64) return set_err(BBP_ERR_ARG, "chi must be 1..64");
  if (precision != BBP_FP64 && precision != BBP_FP32 && precision != BBP_TF32 && precision != BBP_BF16)
    return set_err(BBP_ERR_ARG, "precision must be BBP_FP64, BBP_TF32, BBP_BF16 or BBP_FP32");
  if (!(alpha >= 0.0 && alpha <= 1.0)) return set_err(BBP_ERR_ARG, "alpha must lie in [0, 1]");
  if (ctx->eng.messages_ready) return set_err(BBP_ERR_STATE, "options must be set before bbp_init_messages");
  int rc = ctx->eng.set_precision(precision == BBP_FP64 ? 0 : 1);
  if (rc) return from(ctx, rc);
  ctx->eng.tc_mode = precision == BBP_TF32 ? 1 : precision == BBP_BF16 ? 2 : 0;
  ctx->eng.drop_graphs();
  ctx->eng.chi = chi;
  ctx->eng.alpha = alpha;
  return BBP_OK;
}

bbp_status bbp_set_hermitise(bbp_ctx* ctx, int on) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  ctx->eng.drop_graphs();
  ctx->eng.hermitise = on != 0;
  return BBP_OK;
}

bbp_status bbp_set_power_iters(bbp_ctx* ctx, int power_iters) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (power_iters < 0 || power_iters > 8) return set_err(BBP_ERR_ARG, "power_iters must be 0..8");
  ctx->eng.drop_graphs();
  if (ctx->eng.precision == 0) ctx->eng.power_iters64 = power_iters;
  else ctx->eng.power_iters = power_iters;
  return BBP_OK;
}

bbp_status bbp_set_execution(bbp_ctx* ctx, int use_graphs, int max_streams) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (max_streams < 1 || max_streams > 64) return set_err(BBP_ERR_ARG, "max_streams must be 1..64");
  ctx->eng.drop_graphs();
  ctx->eng.use_graphs = use_graphs != 0;
  ctx->eng.max_streams = max_streams;
  return BBP_OK;
}

bbp_status bbp_set_fuse_cache(bbp_ctx* ctx, size_t max_bytes) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  ctx->eng.drop_graphs();
  ctx->eng.fuse_cache_max = max_bytes;
  if (ctx->eng.fuse_on_the_fly()) ctx->eng.fused.clear();
  return BBP_OK;
}

bbp_status bbp_init_messages(bbp_ctx* ctx, const double* edge_mats) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  return guarded([&] { return from(ctx, ctx->eng.init_messages(edge_mats)); });
}

bbp_status bbp_iterate(bbp_ctx* ctx, double tol, int max_iter, int* iters_out, double* err_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  return guarded([&] { return from(ctx, ctx->eng.iterate(tol, max_iter, iters_out, err_out)); });
}

bbp_status bbp_expect_local(bbp_ctx* ctx, const double* op, int ns, const int* sites, double* re_out,
                            double* im_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!op || !sites || !re_out || !im_out) return set_err(BBP_ERR_ARG, "NULL argument");
  if (ns != 1 && ns != 2) return set_err(BBP_ERR_ARG, "ns must be 1 or 2");
  return guarded([&]() -> bbp_status {
    bbp::Engine& e = ctx->eng;
    if (!e.partitioned || !e.messages_ready) return set_err(BBP_ERR_STATE, "partition and messages are required first");
    const int d = e.d;
    const int n = e.geom.lat.n_sites();
    if (sites[0] < 0 || sites[0] >= n) return set_err(BBP_ERR_ARG, "site out of range");
    std::vector<std::array<int, 2>> coords;
    std::array<int, 2> k1, k2;
    if (ns == 1) {
      int loc = -1;
      int b = e.geom.home_block(sites[0], &loc);
      coords = {{e.geom.blocks[b].X, e.geom.blocks[b].Y}};
      k1 = {0, loc};
    } else {
      int rc = e.bond_region(sites[0], sites[1], coords, k1, k2);
      if (rc) return from(ctx, rc);
    }
    // ns = 1: the operator itself is inserted (one contraction).  ns = 2: the
    // operator is expanded in the product basis |a0><b0| (x) |a1><b1|, one
    // contraction per nonzero entry (the truncated sweep is not linear in
    // the inserted operator, so the expansion is part of the definition).
    const int dim = ns == 1 ? d : d * d;
    std::vector<std::vector<std::array<int, 2>>> C;
    std::vector<std::vector<std::pair<std::array<int, 2>, const double*>>> O;
    std::vector<double> elem;   // host copies of the inserted d x d operators
    std::vector<double2> w;     // weight of each contraction
    const int nb = ns == 1 ? 1 : d * d * d * d;
    elem.assign((size_t)2 * nb * d * d * 2, 0.0);
    bbp::DBuf dev;
    if (!dev.ensure(sizeof(double) * elem.size() + 256, e.stream)) return set_err(BBP_ERR_OOM, "allocation failed");
    C.push_back(coords);
    O.push_back({});
    if (ns == 1) {
      std::memcpy(elem.data(), op, sizeof(double) * 2 * d * d);
      w.push_back(make_double2(1.0, 0.0));
      C.push_back(coords);
      O.push_back({{k1, (const double*)dev.p}});
    }
    int slot = 0;
    for (int a = 0; a < dim && ns == 2; ++a)
      for (int ap = 0; ap < dim; ++ap) {
        double2 wt = make_double2(op[2 * (a * dim + ap)], op[2 * (a * dim + ap) + 1]);
        if (wt.x == 0.0 && wt.y == 0.0) continue;
        w.push_back(wt);
        std::vector<std::pair<std::array<int, 2>, const double*>> ops;
        int a0 = a / d, a1 = a % d, b0 = ap / d, b1 = ap % d;
        double* E0 = elem.data() + (size_t)slot * d * d * 2;
        double* E1 = elem.data() + (size_t)(slot + 1) * d * d * 2;
        E0[2 * (a0 * d + b0)] = 1.0;
        E1[2 * (a1 * d + b1)] = 1.0;
        ops.push_back({k1, (const double*)dev.p + (size_t)slot * d * d * 2});
        ops.push_back({k2, (const double*)dev.p + (size_t)(slot + 1) * d * d * 2});
        slot += 2;
        C.push_back(coords);
        O.push_back(ops);
      }
    cudaError_t ce = cudaMemcpyAsync(dev.p, elem.data(), sizeof(double) * elem.size(), cudaMemcpyHostToDevice, e.stream);
    if (ce != cudaSuccess) return cuda_status(ce);
    std::vector<double> ls, re, im;
    int rc = e.contract_batch(C, O, ls, re, im);
    if (rc) return from(ctx, rc);
    double den = re[0] * re[0] + im[0] * im[0];
    double sr = 0.0, si = 0.0;
    for (size_t j = 1; j < C.size(); ++j) {
      double sc = std::exp(ls[j] - ls[0]);
      // ratio z_j / z_0
      double rr = (re[j] * re[0] + im[j] * im[0]) / den * sc;
      double ri = (im[j] * re[0] - re[j] * im[0]) / den * sc;
      double2 wt = w[j - 1];
      sr += wt.x * rr - wt.y * ri;
      si += wt.x * ri + wt.y * rr;
    }
    *re_out = sr;
    *im_out = si;
    return BBP_OK;
  });
}

bbp_status bbp_expect_product(bbp_ctx* ctx, const double* op1, const double* op2, int site, int slot, double* re_out,
                              double* im_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!op1 || !op2 || !re_out || !im_out) return set_err(BBP_ERR_ARG, "NULL argument");
  return guarded([&]() -> bbp_status {
    bbp::Engine& e = ctx->eng;
    if (!e.partitioned || !e.messages_ready) return set_err(BBP_ERR_STATE, "partition and messages are required first");
    if (site < 0 || site >= e.geom.lat.n_sites() || slot < 0 || slot > 3) return set_err(BBP_ERR_ARG, "bond out of range");
    std::vector<std::array<int, 2>> coords;
    std::array<int, 2> k1, k2;
    if (int rc = e.bond_region(site, slot, coords, k1, k2)) return from(ctx, rc);
    const int d = e.d;
    bbp::DBuf dev;
    if (!dev.ensure(sizeof(double) * 4 * d * d + 256, e.stream)) return set_err(BBP_ERR_OOM, "allocation failed");
    std::vector<double> host(4 * d * d);
    std::memcpy(host.data(), op1, sizeof(double) * 2 * d * d);
    std::memcpy(host.data() + 2 * d * d, op2, sizeof(double) * 2 * d * d);
    cudaError_t ce = cudaMemcpyAsync(dev.p, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, e.stream);
    if (ce != cudaSuccess) return cuda_status(ce);
    const double* d1 = (const double*)dev.p;
    std::vector<std::vector<std::array<int, 2>>> C = {coords, coords};
    std::vector<bbp::OpList> O = {{}, {{k1, d1}, {k2, d1 + 2 * d * d}}};
    std::vector<double> ls, re, im;
    if (int rc = e.contract_batch(C, O, ls, re, im)) return from(ctx, rc);
    const double den = re[0] * re[0] + im[0] * im[0], sc = std::exp(ls[1] - ls[0]);
    *re_out = (re[1] * re[0] + im[1] * im[0]) / den * sc;
    *im_out = (im[1] * re[0] - re[1] * im[0]) / den * sc;
    return BBP_OK;
  });
}

bbp_status bbp_bond_energies(bbp_ctx* ctx, const int* site_slots, int nbonds, double* e_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!site_slots || !e_out || nbonds < 0) return set_err(BBP_ERR_ARG, "bad arguments");
  return guarded([&]() -> bbp_status {
    bbp::Engine& e = ctx->eng;
    if (!e.partitioned || !e.messages_ready) return set_err(BBP_ERR_STATE, "partition and messages are required first");
    std::vector<std::array<int, 2>> bonds(nbonds);
    for (int b = 0; b < nbonds; ++b) bonds[b] = {site_slots[2 * b], site_slots[2 * b + 1]};
    std::vector<double> out;
    if (int rc = e.bond_energies(bonds, out)) return from(ctx, rc);
    std::copy(out.begin(), out.end(), e_out);
    return BBP_OK;
  });
}

bbp_status bbp_block_rdm(bbp_ctx* ctx, int block, const int* sites, int nsites, double* rdm_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!sites || !rdm_out || (nsites != 1 && nsites != 2)) return set_err(BBP_ERR_ARG, "bad arguments");
  return guarded([&]() -> bbp_status {
    bbp::Engine& e = ctx->eng;
    if (!e.partitioned || !e.messages_ready) return set_err(BBP_ERR_STATE, "partition and messages are required first");
    if (block < 0 || block >= e.geom.n_blocks()) return set_err(BBP_ERR_ARG, "block out of range");
    const bbp::Block& b = e.geom.blocks[block];
    std::array<int, 2> keys[2];
    for (int q = 0; q < nsites; ++q) {
      auto it = std::find(b.gids.begin(), b.gids.end(), sites[q]);
      if (it == b.gids.end()) return set_err(BBP_ERR_ARG, "site not in block");
      keys[q] = {0, (int)(it - b.gids.begin())};
    }
    const int d = e.d;
    const int dim = nsites == 1 ? d : d * d;
    std::vector<std::vector<std::array<int, 2>>> C(1 + dim * dim, std::vector<std::array<int, 2>>{{b.X, b.Y}});
    std::vector<std::vector<std::pair<std::array<int, 2>, const double*>>> O(1 + dim * dim);
    std::vector<double> elem((size_t)dim * dim * nsites * d * d * 2, 0.0);
    bbp::DBuf dev;
    if (!dev.ensure(sizeof(double) * elem.size() + 256, e.stream)) return set_err(BBP_ERR_OOM, "allocation failed");
    for (int a = 0; a < dim; ++a)
      for (int bb = 0; bb < dim; ++bb) {
        const int j = a * dim + bb;
        for (int q = 0; q < nsites; ++q) {
          int ia = nsites == 1 ? a : (q == 0 ? a / d : a % d);
          int ib = nsites == 1 ? bb : (q == 0 ? bb / d : bb % d);
          double* E = elem.data() + ((size_t)j * nsites + q) * d * d * 2;
          E[2 * (ib * d + ia)] = 1.0;   // |ib><ia| gives rho[ia, ib]
          O[1 + j].push_back({keys[q], (const double*)dev.p + ((size_t)j * nsites + q) * d * d * 2});
        }
      }
    cudaError_t ce = cudaMemcpyAsync(dev.p, elem.data(), sizeof(double) * elem.size(), cudaMemcpyHostToDevice, e.stream);
    if (ce != cudaSuccess) return cuda_status(ce);
    std::vector<double> ls, re, im;
    int rc = e.contract_batch(C, O, ls, re, im);
    if (rc) return from(ctx, rc);
    double den = re[0] * re[0] + im[0] * im[0];
    std::vector<double> rho(2 * (size_t)dim * dim);
    double tr_re = 0.0, tr_im = 0.0;
    for (int j = 0; j < dim * dim; ++j) {
      double sc = std::exp(ls[1 + j] - ls[0]);
      rho[2 * j] = (re[1 + j] * re[0] + im[1 + j] * im[0]) / den * sc;
      rho[2 * j + 1] = (im[1 + j] * re[0] - re[1 + j] * im[0]) / den * sc;
      if (j / dim == j % dim) { tr_re += rho[2 * j]; tr_im += rho[2 * j + 1]; }
    }
    double tden = tr_re * tr_re + tr_im * tr_im;
    for (int j = 0; j < dim * dim; ++j) {
      double xr = rho[2 * j], xi = rho[2 * j + 1];
      rdm_out[2 * j] = (xr * tr_re + xi * tr_im) / tden;
      rdm_out[2 * j + 1] = (xi * tr_re - xr * tr_im) / tden;
    }
    return BBP_OK;
  });
}

bbp_status bbp_energy_per_site(bbp_ctx* ctx, double* e_out) {
  if (!ctx || !e_out) return set_err(BBP_ERR_ARG, "NULL argument");
  return guarded([&] { return from(ctx, ctx->eng.energy_per_site(e_out)); });
}

bbp_status bbp_norm(bbp_ctx* ctx, double* log_norm_out) {
  if (!ctx || !log_norm_out) return set_err(BBP_ERR_ARG, "NULL argument");
  return guarded([&] { return from(ctx, ctx->eng.log_norm(log_norm_out)); });
}

bbp_status bbp_get_message(bbp_ctx* ctx, int block, int face, int* k_out, int* shapes_out, double* data_out,
                           size_t cap) {
  if (!ctx || !k_out || !shapes_out || !data_out) return set_err(BBP_ERR_ARG, "NULL argument");
  return guarded([&] { return from(ctx, ctx->eng.get_message(block, face, k_out, shapes_out, data_out, cap)); });
}

bbp_status bbp_core_pmps(bbp_ctx* ctx, int block, const int* core_sites, int ncore, int cap_len, int* len_out,
                         int* shapes_out, int* legs_out, double* data_out, size_t cap, double* logscale_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!core_sites || ncore <= 0 || !len_out || !shapes_out || !legs_out || !data_out || !logscale_out)
    return set_err(BBP_ERR_ARG, "bad arguments");
  return guarded([&]() -> bbp_status {
    bbp::Engine& e = ctx->eng;
    if (!e.partitioned || !e.messages_ready) return set_err(BBP_ERR_STATE, "partition and messages are required first");
    if (block < 0 || block >= e.geom.n_blocks()) return set_err(BBP_ERR_ARG, "block out of range");
    const bbp::Block& b = e.geom.blocks[block];
    std::vector<int> core;
    for (int q = 0; q < ncore; ++q) {
      auto it = std::find(b.gids.begin(), b.gids.end(), core_sites[q]);
      if (it == b.gids.end()) return set_err(BBP_ERR_ARG, "site not in block");
      core.push_back((int)(it - b.gids.begin()));
    }
    std::vector<bbp::TShape> shapes;
    std::vector<std::array<int, 2>> legs;
    std::vector<double2> data;
    double ls = 0.0;
    if (int rc = e.core_pmps(block, core, shapes, legs, data, &ls)) return from(ctx, rc);
    if ((int)shapes.size() > cap_len) return set_err(BBP_ERR_ARG, "shapes buffer too small");
    if (2 * data.size() > cap) return set_err(BBP_ERR_ARG, "output buffer too small");
    *len_out = (int)shapes.size();
    for (size_t q = 0; q < shapes.size(); ++q) {
      shapes_out[3 * q] = shapes[q].l;
      shapes_out[3 * q + 1] = shapes[q].p;
      shapes_out[3 * q + 2] = shapes[q].r;
      legs_out[2 * q] = legs[q][0];
      legs_out[2 * q + 1] = legs[q][1];
    }
    for (size_t k = 0; k < data.size(); ++k) {
      data_out[2 * k] = data[k].x;
      data_out[2 * k + 1] = data[k].y;
    }
    *logscale_out = ls;
    return BBP_OK;
  });
}

bbp_status bbp_core_expect(bbp_ctx* ctx, int block, const int* core_sites, int ncore, const double* ops, int nops,
                           double* re_out, double* im_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!core_sites || ncore < 1 || ncore > 2 || nops < 0 || (nops > 0 && (!ops || !re_out || !im_out)))
    return set_err(BBP_ERR_ARG, "bad arguments");
  return guarded([&]() -> bbp_status {
    bbp::Engine& e = ctx->eng;
    if (!e.partitioned || !e.messages_ready) return set_err(BBP_ERR_STATE, "partition and messages are required first");
    if (block < 0 || block >= e.geom.n_blocks()) return set_err(BBP_ERR_ARG, "block out of range");
    const bbp::Block& b = e.geom.blocks[block];
    std::vector<int> core;
    for (int q = 0; q < ncore; ++q) {
      auto it = std::find(b.gids.begin(), b.gids.end(), core_sites[q]);
      if (it == b.gids.end()) return set_err(BBP_ERR_ARG, "site not in block");
      core.push_back((int)(it - b.gids.begin()));
    }
    return from(ctx, e.core_expect(block, core, ops, nops, re_out, im_out));
  });
}

bbp_status bbp_ite_bond(bbp_ctx* ctx, int site, int slot, const double* gate, int max_sweeps, double tol,
                        double* phi_out, int phi_cap, int* n_phi_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!gate || !phi_out || !n_phi_out || phi_cap < 1 || max_sweeps < 0 || !(tol >= 0.0))
    return set_err(BBP_ERR_ARG, "bad arguments");
  return guarded([&]() -> bbp_status {
    std::vector<double> phi;
    if (int rc = ctx->eng.ite_bond(site, slot, gate, max_sweeps, tol, phi)) return from(ctx, rc);
    const int n = (int)std::min<size_t>(phi.size(), (size_t)phi_cap);
    for (int q = 0; q < n; ++q) phi_out[q] = phi[q];
    *n_phi_out = n;
    return BBP_OK;
  });
}

bbp_status bbp_ite(bbp_ctx* ctx, const double* gates, int ndt, const int* bonds, int nbonds, double bp_tol,
                   int bp_max_iter, int als_sweeps, double* energies_out) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!gates || ndt < 0 || !bonds || nbonds <= 0 || !energies_out || bp_max_iter < 0 || als_sweeps < 0 ||
      !(bp_tol >= 0.0))
    return set_err(BBP_ERR_ARG, "bad arguments");
  return guarded([&]() -> bbp_status {
    return from(ctx, ctx->eng.ite(gates, ndt, bonds, nbonds, bp_tol, bp_max_iter, als_sweeps, energies_out));
  });
}

size_t bbp_footprint_bytes(int lattice, int n_sites, int D, int chi, int bx, int by, int precision) {
  (void)precision;
  const size_t z = 16;
  const size_t blk = (size_t)bx * by * (lattice == BBP_KAGOME ? 3 : 1);
  const size_t nblocks = blk ? (n_sites + blk - 1) / blk : 0;
  const size_t k = lattice == BBP_KAGOME ? 2 * (size_t)bx : (size_t)std::max(bx, by);
  const size_t D2 = (size_t)D * D;
  const size_t msgs = nblocks * 4 * 2 * k * chi * chi * D2 * z;
  const size_t fused = (size_t)n_sites * 4 * D2 * D2 * D2 * D2 * z;
  const size_t seg = (size_t)chi * chi * D2 * std::max(D2, (size_t)chi) * z;
  const size_t work = 16 * (12 * seg + 2 * seg);
  return msgs + fused + work + (size_t)n_sites * 2 * D2 * D2 * z;
}

bbp_status bbp_info(bbp_ctx* ctx, int* n_blocks, int* n_updates, int* n_sites) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (!ctx->eng.partitioned) return set_err(BBP_ERR_STATE, "bbp_partition_blocks must come first");
  if (n_blocks) *n_blocks = ctx->eng.geom.n_blocks();
  if (n_updates) *n_updates = (int)ctx->eng.geom.updates().size();
  if (n_sites) *n_sites = ctx->eng.geom.lat.n_sites();
  return BBP_OK;
}

bbp_status bbp_stats(bbp_ctx* ctx, long long* launches_per_iter, double* flops_per_iter) {
  if (!ctx) return set_err(BBP_ERR_ARG, "ctx is NULL");
  if (launches_per_iter) *launches_per_iter = ctx->eng.launches_per_iter;
  if (flops_per_iter) *flops_per_iter = ctx->eng.flops_per_iter;
  return BBP_OK;
}

const char* bbp_last_error(const bbp_ctx* ctx) {
  (void)ctx;
  return g_err.c_str();
}

void bbp_destroy(bbp_ctx* ctx) {
  if (!ctx) return;
  try {
    if (ctx->eng.stream) cudaStreamSynchronize(ctx->eng.stream);
    delete ctx;
  } catch (...) {
  }
}

// ------------------------------------------------------------ kernel level

bbp_status bbp_k_fuse(const double* t, int d, int D, const int* n, const double* op, const int* perm, double* T,
                      void* stream) {
  if (!t || !n || !perm || !T || d < 1 || D < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  int seen = 0;
  for (int q = 0; q < 4; ++q) {
    if (perm[q] < 0 || perm[q] > 3 || (seen >> perm[q]) & 1) return set_err(BBP_ERR_ARG, "perm is not a permutation");
    seen |= 1 << perm[q];
    if (n[q] != 1 && n[q] != D) return set_err(BBP_ERR_ARG, "n[k] must be 1 or D");
  }
  return cuda_status(bbp::launch_fuse((const double2*)t, d, D, n, (const double2*)op, perm, (double2*)T,
                                      (cudaStream_t)stream));
}

size_t bbp_k_svd_work_bytes(int m, int n) { return (m > 0 && n > 0) ? bbp::svd_work_bytes(m, n) : 0; }

bbp_status bbp_k_svd_trunc(const double* Z, int m, int n, int chi, double* U, double* Rem, void* work, int* status,
                           void* stream) {
  if (!Z || !U || !Rem || !work || !status || m < 1 || n < 1 || chi < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  if (std::min(m, n) > 4096) return set_err(BBP_ERR_ARG, "matrix too large");
  return cuda_status(bbp::launch_svd_trunc((const double2*)Z, m, n, chi, (double2*)U, (double2*)Rem, work, status,
                                           (cudaStream_t)stream));
}

bbp_status bbp_k_svd_trunc_noalloc(const double* Z, int m, int n, int chi, double* U, double* Rem, int* status,
                                   void* stream) {
  if (!Z || !U || !Rem || !status || m < 1 || n < 1 || chi < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  bool too_large = false;
  cudaError_t e = bbp::launch_svd_trunc_noalloc((const double2*)Z, m, n, chi, (double2*)U, (double2*)Rem, status,
                                                (cudaStream_t)stream, &too_large);
  if (too_large)
    return set_err(BBP_ERR_ARG, "matrix needs " + std::to_string(bbp::svd_work_bytes(m, n)) +
                                    " bytes of SVD scratch; the allocation-free entry point holds " +
                                    std::to_string(bbp::noalloc_scratch_bytes()));
  return cuda_status(e);
}

bbp_status bbp_k_svd_stats(const void* work, int m, int n, int* sweeps, long long* rotations, void* stream) {
  if (!work || !sweeps || !rotations || m < 1 || n < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  return cuda_status(bbp::svd_stats(work, m, n, sweeps, rotations, (cudaStream_t)stream));
}

void bbp_ktimer_select(int kernel_class) { bbp::ktimer_select(kernel_class); }

bbp_status bbp_ktimer_read(long long* launches, double* ms, double* flops) {
  if (!launches || !ms || !flops) return set_err(BBP_ERR_ARG, "bad arguments");
  bbp::ktimer_read(launches, ms, flops);
  return BBP_OK;
}

bbp_status bbp_k_tc_gemm(int bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C, long long ldc,
                         int M, int N, int K, float alpha, int* err, void* stream) {
  if (!A || !Bt || !C || !err || M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N)
    return set_err(BBP_ERR_ARG, "bad arguments");
  return cuda_status(bbp::launch_tc_gemm(bf16 != 0, A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err,
                                         (cudaStream_t)stream));
}

bbp_status bbp_k_tc_gemm_tile(int bf16, const void* A, long long lda, const void* Bt, long long ldb, float* C,
                              long long ldc, int M, int N, int K, float alpha, int bn, int group_m, int* err,
                              void* stream) {
  if (!A || !Bt || !C || !err || M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N || group_m < 1 ||
      (bn != 64 && bn != 128 && bn != 256))
    return set_err(BBP_ERR_ARG, "bad arguments");
  if (cudaError_t ae = bbp::init_kernel_attributes()) return cuda_status(ae);
  return cuda_status(bbp::launch_tc_gemm_tile(bf16 != 0, A, lda, Bt, ldb, C, ldc, M, N, K, alpha, err,
                                              (cudaStream_t)stream, bn, group_m));
}

bbp_status bbp_autotune_record(int on) {
  bbp::tc_autotune_record(on != 0);
  return BBP_OK;
}

bbp_status bbp_autotune_run(const char* cache_path, int* n_tuned) {
  int n = 0;
  const cudaError_t e = bbp::tc_autotune(cache_path, &n);
  if (n_tuned) *n_tuned = n;
  if (e == cudaErrorInvalidValue) return set_err(BBP_ERR_ARG, "the tile cache could not be written");
  if (e == cudaErrorLaunchTimeout) return set_err(BBP_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
  return cuda_status(e);
}

bbp_status bbp_autotune_load(const char* cache_path, int* n_loaded) {
  if (!cache_path) return set_err(BBP_ERR_ARG, "bad arguments");
  const int n = bbp::tc_autotune_load(cache_path);
  if (n_loaded) *n_loaded = n < 0 ? 0 : n;
  if (n < 0) return set_err(BBP_ERR_ARG, "the tile cache could not be read");
  return BBP_OK;
}

bbp_status bbp_autotune_info(int* n_entries, int* n_pending, unsigned long long* generation) {
  bbp::tc_autotune_info(n_entries, n_pending);
  if (generation) *generation = bbp::tc_tune_generation();
  return BBP_OK;
}

bbp_status bbp_autotune_clear(void) {
  bbp::tc_autotune_clear();
  return BBP_OK;
}

size_t bbp_k_tc_absorb_bytes(int bf16, int P, int Q, int l, int r) {
  return (P > 0 && Q > 0 && l > 0 && r > 0) ? bbp::tc_absorb_bytes(bf16 != 0, P, Q, l, r) : 0;
}

bbp_status bbp_k_tc_absorb(int bf16, int c64, const void* X, int P, int Q, const void* S, int l, int r, void* R,
                           void* work, int* err, void* stream) {
  if (!X || !S || !R || !work || !err || P < 1 || Q < 1 || l < 1 || r < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  if (c64)
    return cuda_status(bbp::launch_tc_absorb(bf16 != 0, (const float2*)X, P, Q, (const float2*)S, l, r, (float2*)R,
                                             work, err, st));
  return cuda_status(bbp::launch_tc_absorb(bf16 != 0, (const double2*)X, P, Q, (const double2*)S, l, r, (double2*)R,
                                           work, err, st));
}

int bbp_k_panel_cluster(int c64, int m, int n) {
  return bbp::panel_cluster(m, n, c64 ? sizeof(float2) : sizeof(double2));
}

bbp_status bbp_k_panel_qr(int c64, const void* A, int m, int n, void* Q, void* R, int batch, int cluster,
                          void* stream) {
  if (!A || m < 1 || n < 1 || m < n || batch < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  const int cmin = bbp::panel_cluster(m, n, c64 ? sizeof(float2) : sizeof(double2), Q != nullptr);
  if (cmin == 0) return set_err(BBP_ERR_ARG, "panel too large for a 16-CTA cluster");
  if (cluster != 0 && (cluster < cmin || cluster > bbp::kPanelMaxCluster))
    return set_err(BBP_ERR_ARG, "cluster size out of range for this panel");
  if (cudaError_t ae = bbp::init_kernel_attributes()) return cuda_status(ae);
  const long long stride = (long long)m * n;
  if (c64)
    return cuda_status(bbp::launch_panel_qr((const float2*)A, m, n, (float2*)Q, (float2*)R, batch, stride,
                                            (cudaStream_t)stream, cluster));
  return cuda_status(bbp::launch_panel_qr((const double2*)A, m, n, (double2*)Q, (double2*)R, batch, stride,
                                          (cudaStream_t)stream, cluster));
}

size_t bbp_k_svd_work_bytes_rand(int c64, int m, int n, int chi, int tensor_cores) {
  if (m < 1 || n < 1 || chi < 1) return 0;
  return c64 ? bbp::svd_work_bytes_c64(m, n, chi, tensor_cores != 0) : bbp::svd_work_bytes_rand64(m, n, chi);
}

bbp_status bbp_k_svd_trunc_rand(int c64, const void* Z, int m, int n, int chi, void* U, void* Rem, void* work,
                                int* status, int power_iters, int tensor_cores, int* err, void* stream) {
  if (!Z || !U || !Rem || !work || !status || m < 1 || n < 1 || chi < 1 || power_iters < 0 || power_iters > 8)
    return set_err(BBP_ERR_ARG, "bad arguments");
  if (tensor_cores && (!c64 || !err)) return set_err(BBP_ERR_ARG, "tensor_cores needs complex64 data and err");
  if (std::min(m, n) > 4096 || chi > 64) return set_err(BBP_ERR_ARG, "matrix too large");
  if (cudaError_t ae = bbp::init_kernel_attributes()) return cuda_status(ae);
  if (c64)
    return cuda_status(bbp::launch_svd_trunc((const float2*)Z, m, n, chi, (float2*)U, (float2*)Rem, work, status,
                                             (cudaStream_t)stream, power_iters, tensor_cores != 0, err));
  return cuda_status(bbp::launch_svd_trunc_rand64((const double2*)Z, m, n, chi, (double2*)U, (double2*)Rem, work,
                                                  status, (cudaStream_t)stream, power_iters));
}

bbp_status bbp_k_fma_peak(int fp64, int blocks, int iters, void* out, double* flops_out, void* stream) {
  if (!out || !flops_out || blocks < 1 || blocks > (1 << 20) || iters < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  *flops_out = bbp::fma_peak_flops(fp64 != 0, blocks, iters);
  return cuda_status(bbp::launch_fma_peak(fp64 != 0, blocks, iters, out, (cudaStream_t)stream));
}

bbp_status bbp_k_qr(double* A, int m, int n, double* Q, double* R, double* tau, void* stream) {
  if (!A || !Q || !R || !tau || m < 1 || n < 1) return set_err(BBP_ERR_ARG, "bad arguments");
  return cuda_status(bbp::launch_qr((double2*)A, m, n, (double2*)Q, (double2*)R, (double2*)tau, (cudaStream_t)stream));
}

bbp_status bbp_plan_debug(int lattice, int Lx, int Ly, int periodic, int bx, int by, int block, int face, int* out,
                          int cap, int* n_steps_out) {
  return guarded([&]() -> bbp_status {
    if (!out || !n_steps_out) return set_err(BBP_ERR_ARG, "NULL argument");
    bbp::Geometry g;
    std::string err = g.build(lattice, Lx, Ly, periodic != 0, bx, by);
    if (!err.empty()) return set_err(BBP_ERR_TILING, err);
    if (block < 0 || block >= g.n_blocks() || face < 0 || face > 3) return set_err(BBP_ERR_ARG, "block or face out of range");
    bbp::Region R;
    err = bbp::build_region(g, {{g.blocks[block].X, g.blocks[block].Y}}, R);
    if (!err.empty()) return set_err(BBP_ERR_TILING, err);
    bbp::SweepPlan plan;
    err = bbp::compile_sweep(g, R, face, plan);
    if (!err.empty()) return set_err(BBP_ERR_TILING, err);
    const int ns = (int)plan.steps.size();
    if (4 * ns > cap) return set_err(BBP_ERR_ARG, "output buffer too small");
    for (int s = 0; s < ns; ++s) {
      const bbp::SweepNode& nd = plan.nodes[s];
      out[4 * s] = nd.site ? 0 : 1;
      out[4 * s + 1] = nd.site ? nd.gid : nd.msg_dir * 1024 + nd.msg_index;
      out[4 * s + 2] = plan.steps[s].nin;
      out[4 * s + 3] = plan.steps[s].nout;
    }
    *n_steps_out = ns;
    return BBP_OK;
  });
}

bbp_status bbp_core_plan_debug(int lattice, int Lx, int Ly, int periodic, int bx, int by, int block,
                               const int* core_sites, int ncore, int* steps_out, int cap, int* info_out, int* legs_out,
                               int cap_len) {
  return guarded([&]() -> bbp_status {
    if (!core_sites || ncore <= 0 || !steps_out || !info_out || !legs_out) return set_err(BBP_ERR_ARG, "NULL argument");
    bbp::Geometry g;
    std::string err = g.build(lattice, Lx, Ly, periodic != 0, bx, by);
    if (!err.empty()) return set_err(BBP_ERR_TILING, err);
    if (block < 0 || block >= g.n_blocks()) return set_err(BBP_ERR_ARG, "block out of range");
    const bbp::Block& b = g.blocks[block];
    std::vector<int> core;
    for (int q = 0; q < ncore; ++q) {
      auto it = std::find(b.gids.begin(), b.gids.end(), core_sites[q]);
      if (it == b.gids.end()) return set_err(BBP_ERR_ARG, "site not in block");
      core.push_back((int)(it - b.gids.begin()));
    }
    bbp::Region R;
    err = bbp::build_region(g, {{b.X, b.Y}}, R);
    if (!err.empty()) return set_err(BBP_ERR_TILING, err);
    bbp::CorePlan cp;
    err = bbp::compile_core(g, R, core, cp);
    if (!err.empty()) return set_err(BBP_ERR_ARG, err);
    const int nb = (int)cp.bottom.steps.size(), nt = (int)cp.top.steps.size();
    if (4 * (nb + nt) > cap || (int)cp.legs.size() > cap_len) return set_err(BBP_ERR_ARG, "output buffer too small");
    int o = 0;
    for (const bbp::SweepPlan* pl : {&cp.bottom, &cp.top})
      for (size_t s = 0; s < pl->steps.size(); ++s) {
        const bbp::SweepNode& nd = pl->nodes[s];
        steps_out[o++] = nd.site ? 0 : 1;
        steps_out[o++] = nd.site ? nd.gid : nd.msg_dir * 1024 + nd.msg_index;
        steps_out[o++] = pl->steps[s].nin;
        steps_out[o++] = pl->steps[s].nout;
      }
    info_out[0] = nb;
    info_out[1] = nt;
    info_out[2] = (int)cp.bottom.final_labels.size();
    info_out[3] = (int)cp.top.final_labels.size();
    info_out[4] = cp.a;
    info_out[5] = cp.c;
    info_out[6] = (int)cp.legs.size();
    for (size_t q = 0; q < cp.legs.size(); ++q) {
      legs_out[2 * q] = cp.legs[q][0];
      legs_out[2 * q + 1] = cp.legs[q][1];
    }
    return BBP_OK;
  });
}

}  // extern "C"
