// Sweep plan compiler and shape simulation (see plan.h).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace bbp {

namespace {

const double kTwoPi = 6.283185307179586;

double angle_of(const Lattice& lat, P4 a, P4 b) {
  double ax, ay, bx, by;
  lat.real(a, ax, ay);
  lat.real(b, bx, by);
  double t = std::atan2(by - ay, bx - ax);
  t = std::fmod(t, kTwoPi);
  if (t < 0) t += kTwoPi;
  return t;
}

double angle_vec(double x, double y) {
  double t = std::fmod(std::atan2(y, x), kTwoPi);
  if (t < 0) t += kTwoPi;
  return t;
}

void sweep_key(int out_dir, P4 p, long long& depth, long long& lat) {
  switch (out_dir) {
    case TOP: depth = p.v; lat = p.u; break;
    case BOTTOM: depth = -p.v; lat = -p.u; break;
    case RIGHT: depth = p.u; lat = -p.v; break;
    default: depth = -p.u; lat = p.v; break;
  }
}

struct PartialSpec {
  const std::vector<std::array<int, 2>>* skip = nullptr;
  long long stop_depth = 0, stop_lat = 0;
};

std::string compile_impl(const Geometry& g, const Region& R, int out_dir, const PartialSpec* part, SweepPlan& plan);

}  // namespace

void plan_sweep_key(int out_dir, P4 p, long long& depth, long long& lat) { sweep_key(out_dir, p, depth, lat); }

std::string compile_sweep(const Geometry& g, const Region& R, int out_dir, SweepPlan& plan) {
  return compile_impl(g, R, out_dir, nullptr, plan);
}

std::string compile_partial_sweep(const Geometry& g, const Region& R, int out_dir,
                                  const std::vector<std::array<int, 2>>& skip, long long stop_depth,
                                  long long stop_lat, SweepPlan& plan) {
  PartialSpec ps;
  ps.skip = &skip;
  ps.stop_depth = stop_depth;
  ps.stop_lat = stop_lat;
  return compile_impl(g, R, out_dir, &ps, plan);
}

namespace {

std::string compile_impl(const Geometry& g, const Region& R, int out_dir, const PartialSpec* part, SweepPlan& plan) {
  const Lattice& lat = g.lat;
  plan = SweepPlan();
  plan.out_dir = out_dir;
  const int start = opposite(out_dir);
  const int lo = (out_dir + 1) & 3, hi = (out_dir + 3) & 3;
  const bool side_forward = (out_dir == TOP || out_dir == RIGHT);
  const bool chain_forward = (out_dir == TOP || out_dir == LEFT);
  // chain-bond labels follow the region's edge labels
  auto bond_label = [&](int d, int m) { return R.n_labels + d * 100000 + m; };

  std::vector<SweepNode> nodes;
  for (const RSite& rs : R.sites) {
    if (part && std::find(part->skip->begin(), part->skip->end(), std::array<int, 2>{rs.inst, rs.local}) !=
                    part->skip->end())
      continue;
    SweepNode n;
    n.site = true; n.inst = rs.inst; n.local = rs.local; n.gid = rs.gid;
    n.nlegs = 4;
    for (int k = 0; k < 4; ++k) { n.label[k] = rs.label[k]; n.ang[k] = angle_of(lat, rs.pos, rs.nbr[k]); }
    sweep_key(out_dir, rs.pos, n.key_depth, n.key_lat);
    nodes.push_back(n);
  }
  for (int d : {lo, hi}) {
    const auto& E = R.sides[d];
    const int K = (int)E.size();
    double tx = (d == BOTTOM || d == TOP) ? 1.0 : 0.0, ty = 1.0 - tx;
    for (int m = 0; m < K; ++m) {
      SweepNode n;
      n.site = false;
      n.msg_inst = E[m].inst; n.msg_dir = E[m].dir; n.msg_index = E[m].index;
      n.nlegs = 3;
      double mx, my;
      lat.real(E[m].mid, mx, my);
      if (m > 0) {
        double px, py; lat.real(E[m - 1].mid, px, py);
        n.ang[0] = angle_vec(px - mx, py - my);
      } else {
        n.ang[0] = angle_vec(-tx, -ty);
      }
      n.ang[1] = angle_of(lat, E[m].mid, E[m].inner);
      if (m < K - 1) {
        double qx, qy; lat.real(E[m + 1].mid, qx, qy);
        n.ang[2] = angle_vec(qx - mx, qy - my);
      } else {
        n.ang[2] = angle_vec(tx, ty);
      }
      n.label[0] = bond_label(d, m);
      n.label[1] = E[m].label;
      n.label[2] = bond_label(d, m + 1);
      sweep_key(out_dir, E[m].mid, n.key_depth, n.key_lat);
      nodes.push_back(n);
    }
  }
  std::stable_sort(nodes.begin(), nodes.end(), [](const SweepNode& a, const SweepNode& b) {
    if (a.key_depth != b.key_depth) return a.key_depth < b.key_depth;
    return a.key_lat < b.key_lat;
  });
  if (part) {   // the bubble halts before the first node at or after the stop key
    size_t keep = 0;
    while (keep < nodes.size() && (nodes[keep].key_depth < part->stop_depth ||
                                   (nodes[keep].key_depth == part->stop_depth && nodes[keep].key_lat < part->stop_lat)))
      ++keep;
    nodes.resize(keep);
  }

  auto end_label = [&](int d, bool at_start) {
    int K = (int)R.sides[d].size();
    int first = bond_label(d, 0), last = bond_label(d, K);
    if (side_forward) return at_start ? first : last;
    return at_start ? last : first;
  };

  // initial boundary
  std::vector<int> labels;
  labels.push_back(end_label(lo, true));
  const auto& S = R.sides[start];
  std::vector<int> order(S.size());
  std::iota(order.begin(), order.end(), 0);
  if (!chain_forward) std::reverse(order.begin(), order.end());
  for (int q : order) {
    labels.push_back(S[q].label);
    plan.start.push_back({S[q].inst, S[q].dir, S[q].index});
  }
  labels.push_back(end_label(hi, true));
  plan.start_reversed = !chain_forward;

  for (size_t s = 0; s < nodes.size(); ++s) {
    const SweepNode& n = nodes[s];
    std::vector<int> pos;
    for (int k = 0; k < n.nlegs; ++k) {
      auto it = std::find(labels.begin(), labels.end(), n.label[k]);
      if (it != labels.end()) pos.push_back((int)(it - labels.begin()));
    }
    if (pos.empty()) return "a swallowed node has no leg on the boundary";
    std::sort(pos.begin(), pos.end());
    int i = pos.front(), j = pos.back();
    if (j - i + 1 != (int)pos.size()) return "in-legs of a swallowed node are not contiguous";
    int nin = (int)pos.size();
    std::vector<int> ccw(n.nlegs);
    std::iota(ccw.begin(), ccw.end(), 0);
    std::stable_sort(ccw.begin(), ccw.end(), [&](int a, int b) { return n.ang[a] < n.ang[b]; });
    int found = -1;
    for (int s0 = 0; s0 < n.nlegs && found < 0; ++s0) {
      bool ok = true;
      for (int q = 0; q < nin; ++q)
        if (n.label[ccw[(s0 + q) % n.nlegs]] != labels[i + q]) { ok = false; break; }
      if (ok) found = s0;
    }
    if (found < 0) return "in-legs of a swallowed node are not in planar order";
    SweepStep st;
    st.node = (int)s; st.i = i; st.j = j; st.nin = nin; st.nout = n.nlegs - nin;
    for (int q = 0; q < nin; ++q) st.in_leg[q] = ccw[(found + q) % n.nlegs];
    for (int q = 0; q < st.nout; ++q)   // reverse ccw order of the remaining legs
      st.out_leg[q] = ccw[(found + n.nlegs - 1 - q) % n.nlegs];
    std::vector<int> newl;
    for (int q = 0; q < st.nout; ++q) newl.push_back(n.label[st.out_leg[q]]);
    labels.erase(labels.begin() + i, labels.begin() + j + 1);
    labels.insert(labels.begin() + i, newl.begin(), newl.end());
    plan.steps.push_back(st);
  }
  if (part) {
    plan.raw = true;
    plan.final_labels = labels;
    plan.nodes = std::move(nodes);
    return "";
  }
  // final boundary
  const auto& O = R.sides[out_dir];
  std::vector<int> want;
  want.push_back(end_label(lo, false));
  if (chain_forward) for (auto& e : O) want.push_back(e.label);
  else for (auto it = O.rbegin(); it != O.rend(); ++it) want.push_back(it->label);
  want.push_back(end_label(hi, false));
  if (want != labels) return "final boundary does not match the out face";
  plan.out_reversed = !chain_forward;
  plan.out_len = (int)O.size();
  plan.nodes = std::move(nodes);
  return "";
}

}  // namespace

std::string compile_core(const Geometry& g, const Region& R, const std::vector<int>& core, CorePlan& cp) {
  cp = CorePlan();
  if (core.empty()) return "the core is empty";
  std::vector<std::array<int, 2>> skip;
  std::vector<const RSite*> cs;
  for (int loc : core) {
    for (const auto& sk : skip)
      if (sk[1] == loc) return "core site repeated";
    const RSite* rs = nullptr;
    for (const RSite& x : R.sites)
      if (x.inst == 0 && x.local == loc) rs = &x;
    if (!rs) return "core site out of range";
    skip.push_back({0, loc});
    cs.push_back(rs);
  }
  long long bd = 0, bl = 0;
  int last = -1;
  for (int k = 0; k < (int)cs.size(); ++k) {
    long long dd, ll;
    sweep_key(TOP, cs[k]->pos, dd, ll);
    if (last < 0 || dd > bd || (dd == bd && ll > bl)) { bd = dd; bl = ll; last = k; }
  }
  long long td, tl;
  sweep_key(BOTTOM, cs[last]->pos, td, tl);
  std::string err = compile_partial_sweep(g, R, TOP, skip, bd, bl, cp.bottom);
  if (err.empty()) err = compile_partial_sweep(g, R, BOTTOM, skip, td, tl, cp.top);
  if (!err.empty()) return err;
  const std::vector<int>& LB = cp.bottom.final_labels;
  const std::vector<int>& LT = cp.top.final_labels;
  const int n = (int)LB.size(), m = (int)LT.size();
  auto in_t = [&](int lab) { return std::find(LT.begin(), LT.end(), lab) != LT.end(); };
  auto in_b = [&](int lab) { return std::find(LB.begin(), LB.end(), lab) != LB.end(); };
  int a = 0;
  while (a < n && in_t(LB[a])) ++a;
  int c = 0;
  while (c < n - a && in_t(LB[n - 1 - c])) ++c;
  if (a == 0 || c == 0 || a + c > m) return "the bubbles do not share both end bonds";
  for (int q = 0; q < a; ++q)
    if (LB[q] != LT[m - 1 - q]) return "the front lines of the bubbles do not match";
  for (int q = 0; q < c; ++q)
    if (LB[n - 1 - q] != LT[q]) return "the front lines of the bubbles do not match";
  for (int q = a; q < n - c; ++q)
    if (in_t(LB[q])) return "a shared leg lies between the core legs";
  for (int q = c; q < m - a; ++q)
    if (in_b(LT[q])) return "a shared leg lies between the core legs";
  if (a >= n - c || c >= m - a) return "the core needs open legs towards both faces";
  cp.a = a;
  cp.c = c;
  auto add = [&](int side, int q, int lab) {
    for (int k = 0; k < (int)cs.size(); ++k)
      for (int sl = 0; sl < 4; ++sl)
        if (cs[k]->label[sl] == lab) {
          cp.ring.push_back({side, q});
          cp.legs.push_back({k, sl});
          return true;
        }
    return false;
  };
  for (int q = a; q < n - c; ++q)
    if (!add(0, q, LB[q])) return "a pMPS leg is not a leg of the core";
  for (int q = c; q < m - a; ++q)
    if (!add(1, q, LT[q])) return "a pMPS leg is not a leg of the core";
  return "";
}

std::string simulate_shapes(const SweepPlan& plan, const LegDims& dims, int chi, ShapeTrace& tr) {
  tr = ShapeTrace();
  std::vector<TShape> A;
  A.push_back(TShape{1, 1, 1});
  for (size_t q = 0; q < plan.start.size(); ++q) {
    TShape s = dims.start[q];
    if (plan.start_reversed) std::swap(s.l, s.r);
    A.push_back(s);
  }
  A.push_back(TShape{1, 1, 1});
  for (size_t q = 0; q + 1 < A.size(); ++q)
    if (A[q].r != A[q + 1].l) return "start chain bond mismatch";
  auto note = [&](const TShape& s) { tr.max_tensor = std::max(tr.max_tensor, s.size()); };
  for (auto& s : A) note(s);
  // right-canonicalise: centre to 0
  for (int p = (int)A.size() - 1; p >= 1; --p) {
    int k = std::min(A[p].l, A[p].p * A[p].r);
    A[p].l = k; A[p - 1].r = k;
  }
  int c = 0;
  tr.max_len = (int)A.size();
  for (const SweepStep& st : plan.steps) {
    ShapeTrace::Step rec;
    while (c < st.i) {
      int k = std::min(A[c].l * A[c].p, A[c].r);
      A[c].r = k; A[c + 1].l = k; ++c; ++rec.moves_qr;
    }
    while (c > st.j) {
      int k = std::min(A[c].l, A[c].p * A[c].r);
      A[c].l = k; A[c - 1].r = k; --c; ++rec.moves_lq;
    }
    const auto& nd = dims.node_dims[st.node];
    int P = 1, Q = 1;
    for (int q = 0; q < st.nin; ++q) {
      int dimq = nd[st.in_leg[q]];
      if (A[st.i + q].p != dimq) return "leg dimension mismatch at a swallow";
      P *= dimq;
    }
    for (int q = 0; q < st.nout; ++q) { rec.out_dims.push_back(nd[st.out_leg[q]]); Q *= nd[st.out_leg[q]]; }
    rec.l = A[st.i].l; rec.r = A[st.j].r; rec.P = P; rec.Q = Q;
    {
      long long pp = 1;   // partial merges of the in-segment
      for (int q = st.i; q <= st.j; ++q) {
        pp *= A[q].p;
        tr.max_seg = std::max(tr.max_seg, (long long)rec.l * pp * A[q].r);
      }
    }
    tr.max_seg = std::max(tr.max_seg, (long long)rec.l * std::max(P, Q) * rec.r);
    std::vector<TShape> nw;
    if (st.nout == 0) {
      if (st.i > 0) {
        A[st.i - 1].r = rec.r;
        A.erase(A.begin() + st.i, A.begin() + st.j + 1);
        c = st.i - 1;
      } else {
        A[st.j + 1].l = rec.l;
        A.erase(A.begin() + st.i, A.begin() + st.j + 1);
        c = st.i;
      }
    } else {
      int l = rec.l;
      long long rest = Q;
      for (int q = 0; q + 1 < st.nout; ++q) {
        rest /= rec.out_dims[q];
        long long rows = (long long)l * rec.out_dims[q], cols = rest * rec.r;
        tr.max_svd_rows = std::max(tr.max_svd_rows, std::min(rows, cols));
        tr.max_svd_cols = std::max(tr.max_svd_cols, std::max(rows, cols));
        int k = (int)std::min<long long>(chi, std::min(rows, cols));
        nw.push_back(TShape{l, rec.out_dims[q], k});
        l = k;
      }
      nw.push_back(TShape{l, rec.out_dims[st.nout - 1], rec.r});
      A.erase(A.begin() + st.i, A.begin() + st.j + 1);
      A.insert(A.begin() + st.i, nw.begin(), nw.end());
      c = st.i + st.nout - 1;
    }
    for (auto& s : nw) note(s);
    rec.split = nw;
    tr.max_len = std::max(tr.max_len, (int)A.size());
    tr.steps.push_back(rec);
  }
  if (plan.raw) {                      // the boundary as it stands, ends included
    tr.final_mps = A;
    return "";
  }
  // merge the two end tensors (both of leg dimension 1)
  if (A.size() < 3) return "final boundary too short";
  A[1].l = A[0].l;
  A[A.size() - 2].r = A.back().r;
  std::vector<TShape> fin(A.begin() + 1, A.end() - 1);
  if (plan.out_reversed) {
    std::reverse(fin.begin(), fin.end());
    for (auto& s : fin) std::swap(s.l, s.r);
  }
  tr.final_mps = fin;
  return "";
}

}  // namespace bbp
