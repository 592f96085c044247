// Union patterns of the node-group tables: the host table builder and the
// node-group kernels (group.cuh) share these definitions.
//
// A group is four consecutive nodes of one grid row.  Take the union of
// their stencil rows in this order:
//   * the nodes of the group's own grid row at offsets RUN0 .. RUN0 + NRUN - 1
//     from the group's first node (along the row, which is periodic on a
//     global grid), then
//   * every other distinct neighbour, by ascending id.
// Every node's stencil row lists its row neighbours at offsets -2, -1, +1,
// +2 first and then the others by ascending id.  A node's terms therefore
// appear in the union in its own row's order, wherever the row neighbours
// fall inside the run.  A kernel that walks the union and applies each entry
// to the nodes whose rows hold it sums every node's terms in the per-node
// order, with the same operations.  It reads each distinct neighbour row
// once for the four nodes, instead of once per node.
//
// A pattern fixes the union's length U and, for every entry, the mask of the
// group's nodes whose rows hold it (bit t for node t of the group).  The
// table builder computes each group's union and compares it with the
// pattern.  Only groups that match entry by entry (masks and run) take the
// union form; every other group keeps per-node rows.  So correctness never
// depends on which patterns exist here, only the speed does.
//
// Away from the octant boundaries of an octahedral reduced Gaussian grid,
// the mesh looks the same around every node.  Each node has two row
// neighbours and two neighbours in each adjacent row; the adjacent rows'
// neighbours of consecutive nodes overlap by one.  So every group in an
// octant's interior has the same union:
//   * one-ring operators: the run -1 .. 4, then five nodes of the row
//     above and five of the row below (U = 16);
//   * the two-ring Laplacian: the run -2 .. 5, then 6, 7, 7 and 6 nodes of
//     the rows two above, one above, one below and two below (U = 34).
// These cover 97% (one-ring) and 96% (Laplacian) of O320's groups, and more
// on finer grids, where the octant boundaries hold a smaller share of the
// nodes.
#pragma once

#if defined(__CUDACC__)
#define ATLASGB_HD __host__ __device__
#else
#define ATLASGB_HD
#endif

namespace atlasgb {
namespace pat {

ATLASGB_HD constexpr int hexval(char c) { return c >= 'a' ? c - 'a' + 10 : c - '0'; }
ATLASGB_HD constexpr int popc4(int m) { return (m & 1) + (m >> 1 & 1) + (m >> 2 & 1) + (m >> 3 & 1); }

// One-ring operators (gradient, divergence, curl, their adjoints, the
// vector gradient).
struct Ring1 {
  static constexpr int U = 16, RUN0 = -1, NRUN = 6;
  ATLASGB_HD static constexpr int mask(int e) { return hexval("125a48136c8136c8"[e]); }
};
// The two-ring Laplacian.
struct Ring2 {
  static constexpr int U = 34, RUN0 = -2, NRUN = 8;
  ATLASGB_HD static constexpr int mask(int e) { return hexval("136db6c8137ec8137fec8137fec8137ec8"[e]); }
};

// Entry e is a node of the group itself (its values are in registers).
template <class P>
ATLASGB_HD constexpr bool in_group(int e) {
  return e < P::NRUN && P::RUN0 + e >= 0 && P::RUN0 + e < 4;
}
// Weights stored before entry e: one set per (entry, node holding it).
template <class P>
ATLASGB_HD constexpr int wbase(int e) {
  int s = 0;
  for (int k = 0; k < e; ++k) s += popc4(P::mask(k));
  return s;
}

}  // namespace pat
}  // namespace atlasgb
