// Dispatch of the shared-memory node-group kernels (group.cuh): storage type
// (FP32, bfloat16) x operator shape x level layout (va, vb).
#include <algorithm>

#include "group.cuh"

namespace atlasgb {
namespace {

constexpr size_t kSmemLimit = 232448;  // 227 KiB of dynamic shared memory per block

template <typename F>
cudaError_t with_shape(const DevTiles& d, F&& f) {
  if (d.nin == 1 && d.nout == 1) return f.template operator()<1, 1, false, 1>();
  if (d.nin == 1 && d.nout == 2 && !d.has_b) return f.template operator()<1, 2, false, 2>();
  if (d.nin == 1 && d.nout == 2) return f.template operator()<1, 2, true, 2>();
  if (d.nin == 2 && d.nout == 1 && d.has_b) return f.template operator()<2, 1, true, 2>();
  return cudaErrorInvalidValue;
}

template <typename S, int NIN, int NOUT, bool HAS_B, int NW, int MODE>
const void* kernel_of(int va, int vb) {
  // entries in flight: merged, four; per-node rows, two steps of four nodes
  constexpr int BATCH = MODE == kTileMerged ? 4 : 2;
  using namespace grp;
#define ATLASGB_TILE(A, B) \
  if (va == A && vb == B) return reinterpret_cast<const void*>(&tile_kernel<S, NIN, NOUT, HAS_B, NW, A, B, BATCH, MODE>);
  ATLASGB_TILE(4, 2)
  ATLASGB_TILE(4, 1)
  ATLASGB_TILE(4, 0)
  ATLASGB_TILE(2, 1)
  ATLASGB_TILE(2, 0)
  ATLASGB_TILE(1, 0)
#undef ATLASGB_TILE
  return nullptr;
}

template <typename S>
struct Pick {
  int va, vb, mode;
  const void* fn = nullptr;
  template <int NIN, int NOUT, bool HAS_B, int NW>
  cudaError_t operator()() {
    fn = mode == kTileMerged ? kernel_of<S, NIN, NOUT, HAS_B, NW, kTileMerged>(va, vb)
                             : kernel_of<S, NIN, NOUT, HAS_B, NW, kTileRows>(va, vb);
    return fn ? cudaSuccess : cudaErrorInvalidValue;
  }
};

const void* tile_fn(StorageType st, const DevTiles& d, int va, int vb) {
  if (st == ST_F32) {
    Pick<float> p{va, vb, d.mode};
    return with_shape(d, p) == cudaSuccess ? p.fn : nullptr;
  }
  if (st == ST_BF16) {
    Pick<uint16_t> p{va, vb, d.mode};
    return with_shape(d, p) == cudaSuccess ? p.fn : nullptr;
  }
  return nullptr;
}

// one field's staged rows (plus slack: the consumers' unconditional loads
// may read up to one level block past a row), the tile table, one stage
void stage_sizes(const DevTiles& d, int64_t ld, int es, size_t& rows, size_t& stage) {
  rows = (static_cast<size_t>(d.max_slots) * static_cast<size_t>(ld) * static_cast<size_t>(es) + 32 * 6 * 4 + 15) &
         ~size_t(15);
  stage = (static_cast<size_t>(d.nin) * rows + static_cast<size_t>(d.max_blob) + 127) & ~size_t(127);
}

}  // namespace

// Stages of a block when bps blocks share an SM: as many as fit (at most
// kMaxStages), at least two (0: two do not fit).
constexpr size_t kSmemPerSM = 233472;  // 228 KiB per SM, 1 KiB of it reserved per block
int stages_for(size_t stage, int bps) {
  const size_t budget = std::min(kSmemLimit, kSmemPerSM / static_cast<size_t>(bps) - 1024);
  int ns = grp::kMaxStages;
  while (ns >= 2 && static_cast<size_t>(ns) * stage + 128 > budget) --ns;
  return ns >= 2 ? ns : 0;
}

size_t tile_smem_bytes(const DevTiles& d, int64_t ld, int elem_size) {
  size_t rows, stage;
  stage_sizes(d, ld, elem_size, rows, stage);
  const int ns = stages_for(stage, 1);
  return ns ? static_cast<size_t>(ns) * stage + 128 : 0;
}

cudaError_t launch_tiles(StorageType st, const DevTiles& d, const TileLaunch& l, cudaStream_t stream) {
  const void* fn = tile_fn(st, d, l.va, l.vb);
  if (!fn) return cudaErrorInvalidValue;
  if (l.ntiles <= 0 || l.nlev <= 0) return cudaSuccess;
  const int es = st == ST_BF16 ? 2 : 4;
  size_t rows, stage;
  stage_sizes(d, l.ld, es, rows, stage);
  // two blocks per SM when asked for and two stages each fit, else one
  int bps = std::max(1, std::min(l.max_bps, 2));
  int ns = stages_for(stage, bps);
  if (ns == 0 && bps == 2) ns = stages_for(stage, bps = 1);
  if (ns == 0) return cudaErrorInvalidValue;
  const size_t smem = static_cast<size_t>(ns) * stage + 128;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  grp::TileArgs a{};
  a.head = d.head;
  a.blob = d.blob;
  a.in0 = l.in0;
  a.in1 = l.in1;
  a.out0 = l.out0;
  a.out1 = l.out1;
  a.t0 = l.t0;
  a.ntiles = l.ntiles;
  a.nlev = l.nlev;
  a.nstore = l.nstore;
  const int lb = 32 * (l.va + l.vb);
  a.nlb = (l.nlev + lb - 1) / lb;
  a.ld = l.ld;
  a.rows_bytes = static_cast<uint32_t>(rows);
  a.stage_bytes = static_cast<uint32_t>(stage);
  a.nstages = ns;
  a.wait_limit = l.wait_limit > 0 ? l.wait_limit : (1ll << 31);  // about a second at 2 GHz
  a.hang_test = l.hang_test;
  void* args[] = {&a};
  const int threads = 32 * (d.groups_per_tile + 1);  // at most 256 (the kernels' launch bound)
  if (threads > 256) return cudaErrorInvalidValue;
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, threads, smem);
  if (e != cudaSuccess) return e;
  bps = std::max(1, std::min(bps, fit));
  const int blocks = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(l.sms) * bps, l.ntiles));
  return cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, stream);
}

cudaError_t tile_error(unsigned* code, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(code, grp::g_tile_error, sizeof(unsigned));
  if (e != cudaSuccess || !clear) return e;
  const unsigned zero = 0u;
  return cudaMemcpyToSymbol(grp::g_tile_error, &zero, sizeof(unsigned));
}

}  // namespace atlasgb
