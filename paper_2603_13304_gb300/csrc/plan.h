// Boundary-MPS sweep plans (host side).
//
// A plan fixes, for one region and one out face, the order in which the
// bubble swallows site tensors and side-message tensors (Sec. 1.1.3), which
// boundary-MPS positions each swallow consumes, and the order of the legs it
// emits.  Rules:
//  * nodes are visited in increasing (depth, lateral) skew coordinates, depth
//    running from the start face (opposite the out face) to the out face;
//  * the boundary MPS starts as [end bond, start-face message, end bond], the
//    end bonds being the start-side ends of the two side-message chains;
//  * a node's legs already on the boundary must be contiguous and appear in
//    counter-clockwise order around the node; its other legs replace them in
//    reverse counter-clockwise order (the planar order of the new boundary);
//  * the sweep ends with [end bond, out-face legs, end bond].
// Shapes follow from the incoming message bond dimensions and chi: a QR/LQ
// move or an SVD split keeps min(rows, cols) (an SVD at most chi) columns.
#pragma once
#include <string>
#include <vector>

#include "geom.h"

namespace bbp {

struct SweepNode {
  bool site = true;
  int inst = -1, local = -1, gid = -1;     // site nodes
  int msg_inst = -1, msg_dir = -1, msg_index = -1;   // message nodes: incoming message tensor
  int nlegs = 0;
  int label[4];
  double ang[4];
  long long key_depth = 0, key_lat = 0;
};

struct SweepStep {
  int node;
  int i, j;          // boundary positions of the in-legs (contiguous)
  int nin, nout;
  int in_leg[4];     // node leg indices, boundary order
  int out_leg[4];    // node leg indices, boundary order
};

struct SweepPlan {
  int out_dir = TOP;
  std::vector<SweepNode> nodes;     // in swallow order
  std::vector<SweepStep> steps;     // steps[s] swallows nodes[s]
  // start chain tensors in boundary (lateral) order: (inst, dir, index)
  std::vector<std::array<int, 3>> start;
  bool start_reversed = false;      // start tensors enter transposed (r, p, l)
  bool out_reversed = false;        // final MPS must be reversed into canonical order
  int out_len = 0;                  // number of out-face legs
  // A bubble that halts before a core (Sec. 2.3, "Core"): the boundary is
  // returned as it stands, end-bond tensors included, in boundary order.
  bool raw = false;
  std::vector<int> final_labels;    // leg label of every boundary position (raw plans)
};

std::string compile_sweep(const Geometry& g, const Region& R, int out_dir, SweepPlan& plan);

// Sweep key of a position for a sweep towards out_dir.
void plan_sweep_key(int out_dir, P4 p, long long& depth, long long& lat);

// A raw plan: the sweep towards out_dir never swallows the sites in `skip`
// (region instance, local index) and halts before the first node whose key
// is (stop_depth, stop_lat) or later.
std::string compile_partial_sweep(const Geometry& g, const Region& R, int out_dir,
                                  const std::vector<std::array<int, 2>>& skip, long long stop_depth,
                                  long long stop_lat, SweepPlan& plan);

// Core extraction (Sec. 2.3, "Core"): the two bubbles around the core sites
// `core` (local indices of the single-block region R) and the structure of
// the zipper that joins them.  The bottom bubble (towards TOP) swallows every
// node before the core's last site in the bottom-up order, the top bubble
// (towards BOTTOM) every node after it; neither swallows the core.  Their
// boundaries share the a leftmost legs of the bottom one (the a rightmost of
// the top one, reversed) and the c rightmost (the c leftmost of the top one);
// the legs between are the core's.  The pMPS takes, in cyclic order, the
// bottom boundary's positions a .. n-c-1, then the top one's c .. m-a-1.
struct CorePlan {
  SweepPlan bottom, top;
  int a = 0, c = 0;
  std::vector<std::array<int, 2>> ring;   // per pMPS tensor: (0 bottom / 1 top, boundary position)
  std::vector<std::array<int, 2>> legs;   // per pMPS tensor: (position in core, slot of that site)
};
std::string compile_core(const Geometry& g, const Region& R, const std::vector<int>& core, CorePlan& cp);

// ---------------------------------------------------------- shape simulation

struct TShape { int l = 1, p = 1, r = 1; long long size() const { return (long long)l * p * r; } };

// Leg dimension of every node leg: site legs -> D^2 (1 on open legs); message
// node legs -> (left bond, D^2, right bond) of the incoming message tensor.
struct LegDims {
  std::vector<std::array<int, 4>> node_dims;   // per plan node
  std::vector<TShape> start;                   // shapes of the start chain tensors (canonical orientation)
};

struct ShapeTrace {
  // per step: the shapes before the step and the segment dims
  struct Step {
    int moves_lq = 0, moves_qr = 0;    // centre moves before the swallow
    int l, r;                          // segment outer bonds
    int P, Q;                          // product of in / out leg dims
    std::vector<int> out_dims;
    std::vector<TShape> split;         // resulting tensors
  };
  std::vector<Step> steps;
  std::vector<TShape> final_mps;       // over the out legs, boundary order, ends merged
  long long max_tensor = 0, max_seg = 0, max_svd_rows = 0, max_svd_cols = 0;
  int max_len = 0;
};

std::string simulate_shapes(const SweepPlan& plan, const LegDims& dims, int chi, ShapeTrace& tr);

}  // namespace bbp
