// Instantiations of the shared-memory node-group kernels for FP32 fields
// (group.cuh): operator shape x level layout (va, vb) x table layout.
#include "group.cuh"

namespace atlasgb {

const void* tile_fn_f32(const DevTiles& d, int va, int vb) {
  grp::Pick<float> p{va, vb};
  return grp::with_shape(d, p) == cudaSuccess ? p.fn : nullptr;
}

}  // namespace atlasgb
