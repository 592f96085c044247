// Launch of the shared-memory node-group kernels (group.cuh); the kernels
// themselves are instantiated per storage type in group_f32.cu and
// group_bf16.cu (compiled in parallel).
#include <algorithm>
#include <mutex>

#include "group.cuh"

namespace atlasgb {
namespace {

constexpr size_t kSmemLimit = 232448;  // 227 KiB of dynamic shared memory per block

const void* tile_fn(StorageType st, const DevTiles& d, const TileLaunch& l) {
  if (l.npw != 4 && l.npw != 2) return nullptr;
  if (st == ST_F32) return tile_fn_f32(d, l.va, l.vb, l.npw);
  if (st == ST_BF16) return tile_fn_bf16(d, l.va, l.vb, l.npw);
  return nullptr;
}

// threads of a block: a consumer warp per part of every group of a tile
// (4 / npw parts of npw nodes per group), then the producer warp
int tile_threads(const DevTiles& d, const TileLaunch& l) { return 32 * ((4 / l.npw) * d.max_groups + 1); }

// The device error word of the tile kernels and its address per device
// (looked up once, with the device current).
__device__ unsigned g_tile_error = 0u;
constexpr int kMaxDevices = 64;
std::mutex g_err_mu;
unsigned* g_err_addr[kMaxDevices] = {};
cudaError_t error_word(unsigned** p) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_addr[dev]) {
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_tile_error);
    if (e != cudaSuccess) return e;
    g_err_addr[dev] = static_cast<unsigned*>(q);
  }
  *p = g_err_addr[dev];
  return cudaSuccess;
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

cudaError_t tile_shape(StorageType st, const DevTiles& d, const TileLaunch& l, int* bps_out, int* stages_out,
                       size_t* smem_out) {
  *bps_out = 0;
  *stages_out = 0;
  *smem_out = 0;
  const void* fn = tile_fn(st, d, l);
  if (!fn) return cudaErrorInvalidValue;
  const int es = st == ST_BF16 ? 2 : 4;
  size_t rows, stage;
  stage_sizes(d, l.ld, es, rows, stage);
  // two blocks per SM when asked for and two stages each fit, else one
  int bps = std::max(1, std::min(l.max_bps, 2));
  int ns = stages_for(stage, bps);
  if (ns == 0 && bps == 2) ns = stages_for(stage, bps = 1);
  if (ns == 0) return cudaSuccess;
  const size_t smem = static_cast<size_t>(ns) * stage + 128;
  const int threads = tile_threads(d, l);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int fit = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, threads, smem);
  if (e != cudaSuccess) return e;
  *bps_out = std::max(1, std::min(bps, fit));
  *stages_out = ns;
  *smem_out = smem;
  return cudaSuccess;
}

cudaError_t launch_tiles(StorageType st, const DevTiles& d, const TileLaunch& l, cudaStream_t stream) {
  const void* fn = tile_fn(st, d, l);
  if (!fn) return cudaErrorInvalidValue;
  if (l.ntiles <= 0 || l.nlev <= 0) return cudaSuccess;
  const int threads = tile_threads(d, l);  // within the kernels' launch bound
  if (threads > tile_max_threads(l.npw, d.nin, d.nout, st == ST_BF16 ? 2 : 4)) return cudaErrorInvalidValue;
  int bps = 0, ns = 0;
  size_t smem = 0;
  cudaError_t e = tile_shape(st, d, l, &bps, &ns, &smem);
  if (e != cudaSuccess) return e;
  if (ns == 0) return cudaErrorInvalidValue;
  const int es = st == ST_BF16 ? 2 : 4;
  size_t rows, stage;
  stage_sizes(d, l.ld, es, rows, stage);
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
  a.wait_hint_ns = l.wait_hint_ns;
  a.bd = l.bd;
  a.bd.nnz = d.blob_words;
  a.max_groups = d.max_groups;
  e = error_word(&a.err);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  const int blocks = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(l.sms) * bps, l.ntiles));
  return cudaLaunchKernel(fn, dim3(blocks), dim3(threads), args, smem, stream);
}

cudaError_t tile_error(unsigned* code, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(code, g_tile_error, sizeof(unsigned));
  if (e != cudaSuccess || !clear) return e;
  const unsigned zero = 0u;
  return cudaMemcpyToSymbol(g_tile_error, &zero, sizeof(unsigned));
}

}  // namespace atlasgb
