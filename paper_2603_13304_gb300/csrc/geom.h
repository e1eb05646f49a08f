// Lattice, block and region geometry for the BlockBP engine (host side).
//
// Blocks follow the tiling rules of Sec. 2.2.2: a block tiles the lattice and
// all edges leaving one face enter the opposite face of one neighbouring block.
// Kagome blocks are the L x L parallelograms of Sec. 2.3.1 (N_T = 3 L^2); the C
// site of the top-left triangle is replaced by its translate C(0,-1) so that
// no bond leaves a corner diagonally, which gives 2L crossing bonds per face.
//
// Coordinates are integer skew coordinates in units of a quarter lattice
// vector; real space is (u, v) for the square lattice and (2u + v, sqrt3 v)
// for the Kagome lattice (a1 = (2, 0), a2 = (1, sqrt 3)).
#pragma once
#include <array>
#include <string>
#include <vector>

namespace bbp {

enum Dir { BOTTOM = 0, RIGHT = 1, TOP = 2, LEFT = 3 };
inline int opposite(int d) { return (d + 2) & 3; }
inline int dir_dx(int d) { return d == RIGHT ? 1 : d == LEFT ? -1 : 0; }
inline int dir_dy(int d) { return d == TOP ? 1 : d == BOTTOM ? -1 : 0; }

struct P4 { int u = 0, v = 0; };

struct Lattice {
  int kind = 0;          // 0 square, 1 kagome
  int Lx = 0, Ly = 0;    // unit cells
  bool periodic = false;
  int ntypes() const { return kind == 0 ? 1 : 3; }
  int n_sites() const { return ntypes() * Lx * Ly; }
  P4 pos4(int t, int i, int j) const;
  void real(P4 p, double& x, double& y) const;
  bool inside(int i, int j) const { return i >= 0 && i < Lx && j >= 0 && j < Ly; }
  int site_id(int t, int i, int j) const;   // -1 outside an open lattice
  // neighbour through slot k: type, i, j, slot
  void neighbour(int t, int i, int j, int k, int& t2, int& i2, int& j2, int& k2) const;
};

struct Edge {        // a leg of a block site that crosses a block face
  int site, slot;    // local site index, its slot
  int gid, gslot;    // neighbour global site id (-1 open) and slot
  P4 inner, outer;
  P4 mid() const { return P4{(inner.u + outer.u) / 2, (inner.v + outer.v) / 2}; }
};

struct Face {
  int nbr = -1;                 // neighbouring block id, -1 open boundary
  std::vector<Edge> edges;      // canonical order: real x (bottom/top), real y (left/right)
};

struct Block {
  int id, X, Y;
  std::vector<std::array<int, 3>> sites;   // (t, i, j)
  std::vector<int> gids;
  std::vector<P4> pos;
  Face faces[4];
  int local_of(int t, int i, int j) const;
};

struct Geometry {
  Lattice lat;
  int bx = 0, by = 0, NBx = 0, NBy = 0;
  std::vector<Block> blocks;

  // returns empty string on success, else the reason
  std::string build(int kind, int Lx, int Ly, bool periodic, int bx, int by);
  void block_of(int t, int i, int j, int& X, int& Y) const;
  int block_id(int X, int Y) const;        // -1 outside an open lattice
  int n_blocks() const { return NBx * NBy; }
  // (sender, out face) pairs, in block-major order; receiver = (nbr, opposite)
  struct Update { int block, face, recv_block, recv_face; };
  std::vector<Update> updates() const;
  int home_block(int gid, int* local) const;
};

// ---------------------------------------------------------------- regions --

struct RSite {
  int inst, local, gid;
  P4 pos;
  int label[4];        // edge label per slot
  P4 nbr[4];           // position of the neighbour image per slot
};

struct RChainEdge {
  int label;           // crossing-edge label
  P4 mid, inner;
  int inst, dir, index;
};

struct Region {
  std::vector<std::array<int, 2>> coords;   // unwrapped block coordinates per instance
  std::vector<int> ids;                     // block id per instance
  std::vector<std::array<int, 2>> shift;    // unit-cell translation per instance
  std::vector<RSite> sites;
  std::vector<RChainEdge> sides[4];
  std::vector<std::array<int, 2>> side_faces[4];   // (inst, dir), canonical order
  int n_labels = 0;
};

std::string build_region(const Geometry& g, const std::vector<std::array<int, 2>>& coords, Region& out);

}  // namespace bbp
