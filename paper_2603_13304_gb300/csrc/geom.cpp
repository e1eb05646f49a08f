// Geometry of lattices, blocks and regions (see geom.h).
#include "geom.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

namespace bbp {

namespace {
// (type, slot) -> (neighbour type, di, dj, neighbour slot)
const int kSquare[1][4][4] = {{{0, 0, 1, 2}, {0, 1, 0, 3}, {0, 0, -1, 0}, {0, -1, 0, 1}}};
const int kKagome[3][4][4] = {
    {{1, 0, 0, 0}, {2, 0, 0, 0}, {1, -1, 0, 2}, {2, 0, -1, 2}},
    {{0, 0, 0, 0}, {2, 0, 0, 1}, {0, 1, 0, 2}, {2, 1, -1, 3}},
    {{0, 0, 0, 1}, {1, 0, 0, 1}, {0, 0, 1, 3}, {1, -1, 1, 3}},
};
int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
int mod(int a, int b) { int r = a % b; return r < 0 ? r + b : r; }
}  // namespace

P4 Lattice::pos4(int t, int i, int j) const {
  if (kind == 0) return P4{4 * i, 4 * j};
  return P4{4 * i + (t == 1 ? 2 : 0), 4 * j + (t == 2 ? 2 : 0)};
}

void Lattice::real(P4 p, double& x, double& y) const {
  double u = p.u / 4.0, v = p.v / 4.0;
  if (kind == 0) { x = u; y = v; return; }
  x = 2.0 * u + v;
  y = std::sqrt(3.0) * v;
}

int Lattice::site_id(int t, int i, int j) const {
  if (periodic) { i = mod(i, Lx); j = mod(j, Ly); }
  else if (!inside(i, j)) return -1;
  if (kind == 0) return (Ly - 1 - j) * Lx + i;   // row 0 is the top row
  return 3 * (j * Lx + i) + t;
}

void Lattice::neighbour(int t, int i, int j, int k, int& t2, int& i2, int& j2, int& k2) const {
  const int* e = kind == 0 ? kSquare[0][k] : kKagome[t][k];
  t2 = e[0]; i2 = i + e[1]; j2 = j + e[2]; k2 = e[3];
}

int Block::local_of(int t, int i, int j) const {
  for (size_t n = 0; n < sites.size(); ++n)
    if (sites[n][0] == t && sites[n][1] == i && sites[n][2] == j) return (int)n;
  return -1;
}

void Geometry::block_of(int t, int i, int j, int& X, int& Y) const {
  if (lat.kind == 1 && t == 2 && mod(i, bx) == 0 && mod(j, by) == by - 1) {
    X = floordiv(i, bx); Y = floordiv(j, by) + 1;   // re-homed corner C site
    return;
  }
  X = floordiv(i, bx); Y = floordiv(j, by);
}

int Geometry::block_id(int X, int Y) const {
  if (lat.periodic) return mod(Y, NBy) * NBx + mod(X, NBx);
  if (X < 0 || X >= NBx || Y < 0 || Y >= NBy) return -1;
  return Y * NBx + X;
}

int Geometry::home_block(int gid, int* local) const {
  for (const Block& b : blocks)
    for (size_t n = 0; n < b.gids.size(); ++n)
      if (b.gids[n] == gid) { if (local) *local = (int)n; return b.id; }
  return -1;
}

std::string Geometry::build(int kind, int Lx, int Ly, bool periodic, int bx_, int by_) {
  if (kind != 0 && kind != 1) return "unknown lattice kind";
  if (Lx <= 0 || Ly <= 0 || bx_ <= 0 || by_ <= 0) return "sizes must be positive";
  if (Lx % bx_ || Ly % by_) return "block size must divide the lattice";
  if (kind == 1 && (bx_ != by_ || bx_ < 2)) return "Kagome blocks are L x L parallelograms with L >= 2";
  if (kind == 1 && !periodic) return "Kagome lattices are periodic super-cells";
  lat.kind = kind; lat.Lx = Lx; lat.Ly = Ly; lat.periodic = periodic;
  bx = bx_; by = by_; NBx = Lx / bx; NBy = Ly / by;
  blocks.clear();
  const int tord_k[3] = {2, 0, 1};   // Up (C), Down-Left (A), Down-Right (B)
  for (int Y = 0; Y < NBy; ++Y)
    for (int X = 0; X < NBx; ++X) {
      Block b;
      b.id = Y * NBx + X; b.X = X; b.Y = Y;
      for (int j = Y * by - 1; j < (Y + 1) * by + 1; ++j)
        for (int i = X * bx - 1; i < (X + 1) * bx + 1; ++i)
          for (int q = 0; q < lat.ntypes(); ++q) {
            int t = kind == 1 ? tord_k[q] : 0;
            int X2, Y2;
            block_of(t, i, j, X2, Y2);
            if (X2 != X || Y2 != Y) continue;
            if (!periodic && !lat.inside(i, j)) continue;
            b.sites.push_back({t, i, j});
            b.gids.push_back(lat.site_id(t, i, j));
            b.pos.push_back(lat.pos4(t, i, j));
          }
      for (size_t n = 0; n < b.sites.size(); ++n) {
        int t = b.sites[n][0], i = b.sites[n][1], j = b.sites[n][2];
        for (int k = 0; k < 4; ++k) {
          int t2, i2, j2, k2;
          lat.neighbour(t, i, j, k, t2, i2, j2, k2);
          if (b.local_of(t2, i2, j2) >= 0) continue;
          int X2, Y2;
          block_of(t2, i2, j2, X2, Y2);
          int dx = X2 - X, dy = Y2 - Y;
          int d = -1;
          if (dx == 0 && dy == -1) d = BOTTOM;
          else if (dx == 1 && dy == 0) d = RIGHT;
          else if (dx == 0 && dy == 1) d = TOP;
          else if (dx == -1 && dy == 0) d = LEFT;
          if (d < 0) return "a bond leaves a block diagonally";
          Edge e;
          e.site = (int)n; e.slot = k;
          e.gid = lat.site_id(t2, i2, j2); e.gslot = k2;
          e.inner = b.pos[n]; e.outer = lat.pos4(t2, i2, j2);
          b.faces[d].edges.push_back(e);
          if (e.gid >= 0) {
            int nb = block_id(X2, Y2);
            if (b.faces[d].nbr < 0) b.faces[d].nbr = nb;
            else if (b.faces[d].nbr != nb) return "a face touches two blocks";
          }
        }
      }
      for (int d = 0; d < 4; ++d) {
        auto& E = b.faces[d].edges;
        std::stable_sort(E.begin(), E.end(), [&](const Edge& a, const Edge& c) {
          double xa, ya, xc, yc;
          lat.real(a.mid(), xa, ya);
          lat.real(c.mid(), xc, yc);
          return (d == BOTTOM || d == TOP) ? xa < xc : ya < yc;
        });
        bool any_open = false, any_conn = false;
        for (auto& e : E) (e.gid < 0 ? any_open : any_conn) = true;
        if (any_open && any_conn) return "a face mixes open and connected edges";
      }
      blocks.push_back(std::move(b));
    }
  return "";
}

std::vector<Geometry::Update> Geometry::updates() const {
  std::vector<Update> out;
  for (const Block& b : blocks)
    for (int d = 0; d < 4; ++d)
      if (b.faces[d].nbr >= 0) out.push_back({b.id, d, b.faces[d].nbr, opposite(d)});
  return out;
}

std::string build_region(const Geometry& g, const std::vector<std::array<int, 2>>& coords, Region& R) {
  const Lattice& lat = g.lat;
  R = Region();
  R.coords = coords;
  std::map<std::pair<int, int>, int> where;
  for (size_t n = 0; n < coords.size(); ++n) {
    where[{coords[n][0], coords[n][1]}] = (int)n;
    int bid = g.block_id(coords[n][0], coords[n][1]);
    if (bid < 0) return "region block outside the lattice";
    const Block& b = g.blocks[bid];
    R.ids.push_back(bid);
    R.shift.push_back({(coords[n][0] - b.X) * g.bx, (coords[n][1] - b.Y) * g.by});
  }
  // labels: internal edges first (by sorted endpoint triple), then crossing edges
  std::map<std::tuple<int, int, int, int, int, int>, int> internal;
  std::map<std::tuple<int, int, int>, int> crossing;
  std::vector<RSite> sites;
  struct Pending { size_t site; int k; bool internal_edge; std::tuple<int, int, int, int, int, int> key; std::tuple<int, int, int> xkey; };
  std::vector<Pending> pend;
  for (size_t n = 0; n < coords.size(); ++n) {
    const Block& b = g.blocks[R.ids[n]];
    int tx = R.shift[n][0], ty = R.shift[n][1];
    for (size_t loc = 0; loc < b.sites.size(); ++loc) {
      int t = b.sites[loc][0], i = b.sites[loc][1] + tx, j = b.sites[loc][2] + ty;
      RSite rs;
      rs.inst = (int)n; rs.local = (int)loc; rs.gid = b.gids[loc];
      rs.pos = lat.pos4(t, i, j);
      for (int k = 0; k < 4; ++k) {
        int t2, i2, j2, k2;
        lat.neighbour(t, i, j, k, t2, i2, j2, k2);
        rs.nbr[k] = lat.pos4(t2, i2, j2);
        int X2, Y2;
        g.block_of(t2, i2, j2, X2, Y2);
        auto it = where.find({X2, Y2});
        Pending p;
        p.site = sites.size(); p.k = k;
        if (it != where.end() && (lat.periodic || lat.inside(i2, j2))) {
          int m = it->second;
          const Block& b2 = g.blocks[R.ids[m]];
          int loc2 = b2.local_of(t2, i2 - R.shift[m][0], j2 - R.shift[m][1]);
          if (loc2 < 0) return "region neighbour not found";
          auto a = std::make_tuple((int)n, (int)loc, k);
          auto c = std::make_tuple(m, loc2, k2);
          if (c < a) std::swap(a, c);
          p.internal_edge = true;
          p.key = std::tuple_cat(a, c);
        } else {
          p.internal_edge = false;
          p.xkey = std::make_tuple((int)n, (int)loc, k);
        }
        pend.push_back(p);
      }
      sites.push_back(rs);
    }
  }
  for (auto& p : pend)
    if (p.internal_edge && !internal.count(p.key)) { int id = (int)internal.size(); internal[p.key] = id; }
  int n_int = (int)internal.size();
  for (auto& p : pend)
    if (!p.internal_edge && !crossing.count(p.xkey)) { int id = n_int + (int)crossing.size(); crossing[p.xkey] = id; }
  for (auto& p : pend)
    sites[p.site].label[p.k] = p.internal_edge ? internal[p.key] : crossing[p.xkey];
  R.sites = std::move(sites);
  R.n_labels = n_int + (int)crossing.size();

  for (int d = 0; d < 4; ++d) {
    struct Entry { double key; int n; std::vector<RChainEdge> edges; };
    std::vector<Entry> entries;
    for (size_t n = 0; n < coords.size(); ++n) {
      if (where.count({coords[n][0] + dir_dx(d), coords[n][1] + dir_dy(d)})) continue;
      const Block& b = g.blocks[R.ids[n]];
      P4 off = lat.pos4(0, R.shift[n][0], R.shift[n][1]);
      Entry en;
      en.n = (int)n;
      const auto& E = b.faces[d].edges;
      for (size_t idx = 0; idx < E.size(); ++idx) {
        RChainEdge ce;
        ce.inner = P4{E[idx].inner.u + off.u, E[idx].inner.v + off.v};
        P4 outer{E[idx].outer.u + off.u, E[idx].outer.v + off.v};
        ce.mid = P4{(ce.inner.u + outer.u) / 2, (ce.inner.v + outer.v) / 2};
        ce.label = crossing.at(std::make_tuple((int)n, E[idx].site, E[idx].slot));
        ce.inst = (int)n; ce.dir = d; ce.index = (int)idx;
        en.edges.push_back(ce);
      }
      double x, y;
      lat.real(en.edges.front().mid, x, y);
      en.key = (d == BOTTOM || d == TOP) ? x : y;
      entries.push_back(std::move(en));
    }
    std::stable_sort(entries.begin(), entries.end(), [](const Entry& a, const Entry& b) { return a.key < b.key; });
    for (auto& en : entries) {
      for (auto& ce : en.edges) R.sides[d].push_back(ce);
      R.side_faces[d].push_back({en.n, d});
    }
  }
  return "";
}

}  // namespace bbp
