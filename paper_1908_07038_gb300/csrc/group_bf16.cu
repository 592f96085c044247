// Instantiations of the shared-memory node-group kernels for bfloat16 fields
// (group.cuh): operator shape x level layout (va, vb) x table layout.
#include "group.cuh"

namespace atlasgb {

const void* tile_fn_bf16(const DevTiles& d, int va, int vb) {
  grp::Pick<uint16_t> p{va, vb};
  return grp::with_shape(d, p) == cudaSuccess ? p.fn : nullptr;
}

}  // namespace atlasgb
