// Launch interface between the C ABI (capi.cpp) and the CUDA kernels
// (kernels.cu, group.cu).  Plain structs of device pointers; no CUDA types leak into
// the C ABI header.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace atlasgb {

enum StorageType { ST_F32 = 0, ST_F64 = 1, ST_BF16 = 2 };

// Branch-free division of 32-bit unsigned integers by a divisor fixed per
// launch: q = (t + ((n - t) >> s1)) >> s2 with t = umulhi(m, n).
struct Div32 {
  uint32_t m;
  uint32_t s1, s2;
};

// Index bounds of one launch, checked by the kernels of the bounds-checked
// build (ATLASGB_BOUNDSCHECK; see bounds.cuh) and ignored otherwise: input
// rows [lo, hi) and output rows [olo, ohi) in global node ids, table entries
// [0, nnz) (CSR entries, edges or source nodes, by kernel), and the device
// word pair {code, index} the first violation is recorded in.
struct Bounds {
  int32_t lo = 0, hi = 0, olo = 0, ohi = 0;
  int64_t nnz = 0;
  unsigned long long* err = nullptr;
};
// The device word pair of the bounds checks on the current device (looked
// up once per device), and a synchronous read of it (with clear, reset).
unsigned long long* bounds_word();
cudaError_t bounds_error(unsigned long long* code, long long* index, bool clear);
// Whether this library was built with the kernels' bounds checks.
bool bounds_checked();

// Device tables of one node stencil (see Stencil in geometry.h).  One-input
// operators with float weights (F32 and BF16 fields): w holds packed entries
// {j, w} (scalar_w) or {j, w0, w1, 0} as 32-bit words and nbr is unused.
// Otherwise nbr[nnz] and w[nnz] (scalar_w) or w[nnz][2] in the weight
// precision (double for F64 fields).  b holds [V][2], or is null.
struct DevStencil {
  const int32_t* ptr = nullptr;
  const int32_t* nbr = nullptr;
  const void* w = nullptr;
  const void* b = nullptr;
  int32_t nnodes = 0;
  int64_t nnz = 0;
  int nin = 1, nout = 1;
  bool has_b = false, scalar_w = false;
};

struct StencilLaunch {
  const void* in0 = nullptr;
  const void* in1 = nullptr;
  void* out0 = nullptr;
  void* out1 = nullptr;
  int32_t nlev = 0;
  int64_t ld = 0;
  int vec = 1;
  int batch = 6;   // CSR entries whose neighbour values are requested together (3 or 6)
  int threads = 256;
  int blocks = 0;  // grid size
  uint32_t tile = 0;  // items per block tile: a multiple of threads, blocks * tile < 2^31
  // nodes computed: node0 .. node0 + count - 1.  The
  // field pointers are indexed with global node ids within that range and
  // its neighbours.
  int32_t node0 = 0;
  int32_t count = 0;
  Bounds bd;
};

// Shared-memory node-group kernels (group.cu; tables as TileStencil in
// geometry.h): tile heads int32 [ntiles][kTileHead] and the per-tile table
// blob.  The kernels run on tiles t0 .. t0 + ntiles - 1 with one producer
// warp and one consumer warp per group of a tile.
struct DevTiles {
  const int32_t* head = nullptr;
  const uint32_t* blob = nullptr;
  int32_t ntiles = 0;
  int32_t max_slots = 0;  // most node rows a tile stages
  int32_t max_blob = 0;   // largest tile table (bytes)
  int64_t blob_words = 0; // 32-bit words of blob
  int groups_per_tile = 8;
  int max_groups = 8;        // most groups any tile holds (sets the consumer warps)
  int nin = 1, nout = 1, nw = 1;
  bool has_b = false;
  bool unions = false;       // union groups present: one warp per group only
  int64_t union_groups = 0;  // groups stored in union form
};
struct TileLaunch {
  const void* in0 = nullptr;
  const void* in1 = nullptr;
  void* out0 = nullptr;
  void* out1 = nullptr;
  int32_t nlev = 0;
  int32_t nstore = 0;  // stores cover levels < nstore (nlev rounded up to the row's vector width)
  int64_t ld = 0;      // ld * element size must be a multiple of 16, the field pointers 16-byte aligned
  int va = 4, vb = 1;  // levels per lane in part A and part B of a level block
  int npw = 4;         // nodes per consumer warp: 4 (a warp per group) or 2 (two warps per group)
  int32_t t0 = 0, ntiles = 0;
  int sms = 1;         // grid: sms * (blocks that fit per SM, at most 2), at most ntiles
  int max_bps = 2;
  long long wait_limit = 0;  // clock cycles a wait may take (0: the default, about one second)
  int hang_test = 0;         // 1: the consumers wait on a barrier nothing completes (tests the time-out)
  uint32_t wait_hint_ns = 0; // suspension hint of the consumers' barrier waits (0: none)
  Bounds bd;                 // input rows, output rows; nnz: the blob's 32-bit words
};
// Valid (va, vb) pairs: (1,0) (2,0) (2,1) (4,0) (4,1) (4,2).
// Threads a node-group block may have (the kernels' launch bound): 384 with
// four nodes per warp (up to 11 groups per tile), 512 with two (up to 7).
// Launch bound of the node-group kernels.  Each of an SM's four schedulers
// holds a quarter of the register file, so 12 warps (three per scheduler)
// can have up to 168 registers and 16 warps up to 128.  With one warp per
// group: 384 threads (eleven groups and the producer) for the one-ring
// shapes, which need about 150 registers, and 512 (fifteen groups) for the
// one-input one-output Laplacian and the one-input bfloat16 shapes, which
// need no more than 128.  With two warps per group, 512.
inline int tile_max_threads(int npw, int nin, int nout, int elem_size) {
  return npw == 4 ? ((nin == 1 && nout == 1) || (nin == 1 && elem_size == 2) ? 512 : 384) : 512;
}
constexpr int kTileMaxGroups = 15;  // groups per tile the tables may hold
cudaError_t launch_tiles(StorageType st, const DevTiles& d, const TileLaunch& l, cudaStream_t stream);
// Dynamic shared memory one block needs (two stages), or 0 above the limit.
size_t tile_smem_bytes(const DevTiles& d, int64_t ld, int elem_size);
// The launch shape launch_tiles would take: blocks per SM, stages per block
// and dynamic shared memory per block (0s when the tiles do not fit).
cudaError_t tile_shape(StorageType st, const DevTiles& d, const TileLaunch& l, int* bps, int* stages, size_t* smem);
// Read (and with clear, reset) the device error word of the tile kernels
// (a synchronous copy).
cudaError_t tile_error(unsigned* code, bool clear);

// Edge-based two-pass data on the device.
struct DevEdges {
  const int32_t* e2n = nullptr;   // [E][2]
  const void* coef = nullptr;     // [E][3] (k1, k2, k3) in the weight precision
  const int32_t* ptr = nullptr;   // [V+1]
  const int32_t* ent = nullptr;   // [nnz] edge << 1 | negative
  const void* node = nullptr;     // [V][3] (1/V, cos/V, pole coefficient)
  int32_t nnodes = 0;
  int64_t nedges = 0;
  int64_t nent = 0;               // entries of ent
};

// Persistent batched launch: one descriptor per field.
struct BatchDescDev {
  const int32_t* ptr;
  const int32_t* nbr;
  const void* w;
  const void* b;
  const void* in0;
  const void* in1;
  void* out0;
  void* out1;
  int64_t ld;
  int32_t tile0;      // first tile of this descriptor
  int32_t items;      // nnodes * nvec (< 2^31)
  int32_t nlev;
  int32_t nvec;
  int32_t op;         // 0 gradient (1 in, 2 out), 1 divergence (2 in, 1 out, with b)
  uint32_t div_m;     // division by nvec (see Div32)
  uint32_t div_s1, div_s2;
  int32_t nnodes;     // nodes of the field (rows of in0/in1/out0/out1)
  int64_t nnz;        // CSR entries of the table
};
// The whole table travels as one kernel parameter (at most 32 KB).
constexpr int kBatchMaxDesc = 256;
constexpr int kBatchMaxThreads = 256;  // the batch kernel's launch bound
struct BatchParams {
  int32_t ndesc;
  int32_t ntiles;
  int32_t tile_items;
  int32_t pad;
  unsigned long long* err;  // the bounds checks' word pair (bounds-checked build)
  BatchDescDev d[kBatchMaxDesc];
};
static_assert(sizeof(BatchParams) <= 32764, "kernel parameters are limited to 32764 bytes");

cudaError_t launch_stencil(StorageType st, const DevStencil& s, const StencilLaunch& l, cudaStream_t stream);
// Maximum resident blocks per SM of the stencil kernel for this configuration.
int stencil_occupancy(StorageType st, const DevStencil& s, int vec, int batch, int threads);

// The two passes check their tables against the mesh: node ids [0, nnodes),
// edge ids [0, nedges).
cudaError_t launch_edge_flux(StorageType st, int op, const DevEdges& e, const void* in0, const void* in1,
                             void* flux0, void* flux1, int32_t nlev, int64_t ld, int vec, int threads,
                             int blocks, cudaStream_t stream);
cudaError_t launch_node_gather(StorageType st, int op, const DevEdges& e, const void* flux0, const void* flux1,
                               const void* vin, void* out0, void* out1, int32_t nlev, int64_t ld, int vec,
                               int threads, int blocks, cudaStream_t stream);

Div32 make_div32(uint32_t d);

// FP64 rate probe: blocks x threads threads, 8 chains of iters FMAs each.
cudaError_t launch_fp64_fma(double* out, int blocks, int threads, int64_t iters, cudaStream_t stream);

// Library-owned static device scratch (noalloc.cu): its size, and its device
// address on the current device (looked up once per device).
size_t noalloc_scratch_bytes();
cudaError_t noalloc_scratch(void** ptr);
cudaError_t launch_batch(StorageType st, int vec, bool idx32, const BatchParams& params, int threads, int blocks,
                         cudaStream_t stream);
int batch_occupancy(StorageType st, int vec, bool idx32, int threads);

// Remapping by linear interpolation: nodes int4[ntgt] {n0, n1, n2, 0},
// weights A[ntgt][4] (float for F32/BF16 fields, double for F64).
struct RemapLaunch {
  const void* nodes = nullptr;
  const void* weights = nullptr;
  const void* src = nullptr;
  void* dst = nullptr;
  int32_t ntgt = 0, nlev = 0;
  int64_t ld_src = 0, ld_dst = 0;
  int vec = 1;
  bool idx32 = true;
  int threads = 256, blocks = 1;
  Bounds bd;  // source rows [lo, hi)
};
cudaError_t launch_remap(StorageType st, const RemapLaunch& r, cudaStream_t stream);

// Volume-weighted sums I_k = sum_i V_i x_{i,k} (FP64) over count nodes whose
// rows start at x (V already offset to the first node): nblocks blocks of
// chunk nodes write part[nblocks][nlev], then out[nlev].
struct IntegralLaunch {
  const double* V = nullptr;
  const void* x = nullptr;
  int32_t count = 0, chunk = 0, nlev = 0, nblocks = 0;
  int64_t ld = 0;
  double* part = nullptr;
  double* out = nullptr;
};
cudaError_t launch_integral(StorageType st, const IntegralLaunch& l, cudaStream_t stream);

}  // namespace atlasgb
