// Instantiations of the shared-memory node-group kernels for bfloat16 fields
// (group.cuh): operator shape x level layout (va, vb) x nodes per warp.
#include "group.cuh"

namespace atlasgb {

const void* tile_fn_bf16(const DevTiles& d, int va, int vb, int npw) {
  grp::Pick<uint16_t> p{va, vb, npw};
  return grp::with_shape(d, p) == cudaSuccess ? p.fn : nullptr;
}

}  // namespace atlasgb
