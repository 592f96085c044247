// Index checks of the bounds-checked build (compiled with
// -DATLASGB_BOUNDSCHECK).
//
// Every index a kernel takes from a table (a neighbour id, a CSR row range,
// an edge id, a staged slot, a tile's copy range) is checked against the
// bounds its launch was given before it is used.  The first violation of a
// launch sequence is recorded in a device word pair {code, index} (one
// atomic compare-and-swap decides which), and the access is redirected to a
// valid one (the node itself, an empty row), so the kernel runs to its end
// without touching memory outside its buffers; the library call then
// returns ATLAS_EBOUNDS.  In the normal build the checks compile to nothing.
#pragma once

#include <cstdint>

#include "kernels.h"

namespace atlasgb {

// codes recorded in Bounds::err[0]
enum BoundsCode : unsigned {
  BC_NEIGHBOUR = 1,  // a stencil neighbour id outside the input rows (index: the CSR entry)
  BC_ROW = 2,        // a CSR row range outside the table, or decreasing (index: the node)
  BC_EDGE_END = 3,   // an edge end outside the node range (index: the edge)
  BC_EDGE_ID = 4,    // a node->edge entry outside the edge range (index: the entry)
  BC_TILE_HEAD = 5,  // a tile header (copy ranges, sizes) outside its buffers (index: the tile)
  BC_TILE_TABLE = 6, // a tile's group table or slot outside the staged tile (index: the tile)
  BC_OUTPUT = 7,     // an output row outside the written range (index: the node)
  BC_REMAP = 8,      // a remap source node outside the source field (index: the target)
};

#ifdef ATLASGB_BOUNDSCHECK
constexpr bool kBoundsCheck = true;
__device__ __forceinline__ bool in_bounds(bool ok, unsigned long long* err, unsigned code, long long index) {
  if (!ok && err != nullptr && atomicCAS(err, 0ull, static_cast<unsigned long long>(code)) == 0ull)
    err[1] = static_cast<unsigned long long>(index);
  return ok;
}
#else
constexpr bool kBoundsCheck = false;
__device__ __forceinline__ bool in_bounds(bool, unsigned long long*, unsigned, long long) { return true; }
#endif

}  // namespace atlasgb
