// Cluster tree and block partition of the H-matrix far field (host side; hmatrix_tree.cpp).
//
// Both are pure index work on the mesh: the same rules, evaluated in the same IEEE double
// operations, give the same tree on every machine.  hmatrix_tree.cpp is compiled without
// floating-point contraction so that no fused multiply-add changes a comparison.
#pragma once

#include <stdint.h>

#include <vector>

namespace bem {
namespace hm {

struct Tree {
  std::vector<int32_t> perm;          // tree position -> element
  std::vector<int32_t> begin, size;   // per cluster: first position in perm, number of elements
  std::vector<int32_t> left, right;   // per cluster: children (-1 for a leaf)
  std::vector<double> lo, hi;         // per cluster: vertex bounding box (3 each)
  std::vector<double> diam;           // per cluster: bounding-box diagonal
  int64_t n() const { return (int64_t)begin.size(); }
  bool leaf(int32_t c) const { return left[c] < 0; }
};

struct Partition {
  std::vector<int32_t> lowrank;  // pairs (target cluster, source cluster)
  std::vector<int32_t> dense;
};

// Recursive median bisection along the longest side of the centroids' bounding box (lowest axis
// on ties), elements ordered by that coordinate and then by index, size / 2 to the left, until
// a cluster holds at most `leaf` elements.  Clusters in depth-first order.
void cluster_tree(const double* verts, int64_t nv, const int32_t* tris, int64_t ne, int leaf, Tree& t);

// Depth-first subdivision of (root, root): low-rank block when both sizes <= max_block and
// max(diam) <= eta dist of the bounding boxes (dist > 0); dense block when both are leaves;
// otherwise both sides split (only the non-leaf side when one is a leaf), target children outer.
void block_partition(const Tree& t, double eta, int max_block, Partition& p);

}  // namespace hm
}  // namespace bem
