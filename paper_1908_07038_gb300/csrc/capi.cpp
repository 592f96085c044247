// C ABI of libatlasgb.so (declared in include/atlas_gb.h): handles,
// argument validation, table upload and kernel dispatch.  Every compute call
// runs on the GPU; without a CUDA device the operator calls fail.
#include "atlas_gb.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "geometry.h"
#include "kernels.h"

using atlasgb::StorageType;

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string g_err;

// NVTX range over one library call: visible to profilers (ncu --nvtx, Nsight
// Systems), a no-op otherwise (NVTX is header-only and does nothing unless a
// tool is attached).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
  CallRange(const CallRange&) = delete;
  CallRange& operator=(const CallRange&) = delete;
};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  if (std::getenv("ATLAS_DEBUG")) std::fprintf(stderr, "[atlas error] %s\n", buf);
  return code;
}
int ok() {
  g_err.clear();
  return ATLAS_OK;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(ATLAS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Bounds-checked build: wait for the stream and turn an index violation a
// kernel recorded into ATLAS_EBOUNDS (a stream being captured into a graph
// is not waited for).  The normal build returns at once.
int bounds_after(void* stream, const char* what) {
  if (!atlasgb::bounds_checked()) return ATLAS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return ATLAS_OK;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, what);
  unsigned long long code = 0;
  long long index = 0;
  e = atlasgb::bounds_error(&code, &index, true);
  if (e != cudaSuccess) return cuda_fail(e, "reading the bounds-check word");
  if (code != 0)
    return fail(ATLAS_EBOUNDS, "%s: bounds check %llu failed at index %lld (the access was skipped)", what, code,
                index);
  return ATLAS_OK;
}

std::mutex g_registry_mu;
std::set<const void*> g_live;  // live handles of every kind

void reg(const void* h) {
  std::lock_guard<std::mutex> lk(g_registry_mu);
  g_live.insert(h);
}
bool live(const void* h) {
  std::lock_guard<std::mutex> lk(g_registry_mu);
  return h != nullptr && g_live.count(h) != 0;
}
void unreg(const void* h) {
  std::lock_guard<std::mutex> lk(g_registry_mu);
  g_live.erase(h);
}
}  // namespace

// ----------------------------------------------------------------- handles
struct atlas_grid_s {
  atlasgb::Grid g;
  int users = 0;
};
struct atlas_mesh_s {
  atlas_grid_s* grid = nullptr;
  atlasgb::Mesh m;
  int users = 0;
};

namespace {
// Testing hook (atlas_debug_fail_allocations): the number of device
// allocations still allowed before the next ones fail, or -1 (never fail).
std::atomic<int64_t> g_alloc_budget{-1};

struct DevAlloc {
  std::vector<void*> ptrs;
  template <typename T>
  T* upload(const std::vector<T>& h, cudaError_t& err) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
    int64_t left = g_alloc_budget.load();
    while (left >= 0) {  // consume one allowed allocation, or fail
      if (left == 0) {
        err = cudaErrorMemoryAllocation;
        return nullptr;
      }
      if (g_alloc_budget.compare_exchange_weak(left, left - 1)) break;
    }
    err = cudaMalloc(&p, bytes);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    if (!h.empty()) err = cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

template <typename A>
std::vector<A> convert(const std::vector<double>& v) {
  std::vector<A> out(v.size());
  for (size_t k = 0; k < v.size(); ++k) out[k] = static_cast<A>(v[k]);
  return out;
}

// Tile tables of one operator for the shared-memory node-group kernels
// (FP32 and BF16 fields): built with the per-node tables when the stencil
// allows (ascending rows, node ids below 2^28, few row runs per tile), else
// absent and the per-node kernels run.
struct GroupTables {
  bool ok = false;
  atlasgb::DevTiles dev;
  DevAlloc mem;
  std::vector<int64_t> first;      // first node of every unit (runs of whole grid rows), then nnodes
  std::vector<int32_t> unit_tile;  // first tile of every unit, then ntiles
  int groups = 0;                  // groups per tile the tables were cut with
  int rows = 1;                    // grid rows per tile
  bool unions = false;             // groups matching their union pattern stored in union form
};
struct OpTables {
  bool ready = false;
  atlasgb::DevStencil dev;
  DevAlloc mem;
  GroupTables grp;
};
struct EdgeTables {
  bool ready = false;
  atlasgb::DevEdges dev;
  DevAlloc mem;
};
struct LaunchCfg {
  int vec = 0;  // 0 = widest the dtype and alignment allow
  int batch = 6;
  int threads = 128;
  int blocks_per_sm = 0;  // 0 = occupancy limit
  int tile_passes = 1;    // block tile = tile_passes * threads items (1 = grid-stride loop)
  int group = 1;          // node-group kernel: 1 where it applies and pays (tile_min_levels), 2 wherever it applies, 0 never
  int tile_bps = 1;       // node-group kernel: blocks per SM at most (1 or 2; fewer when shared memory is short)
  int tile_groups = 7;    // node-group kernel: groups of four nodes per tile (1..kTileMaxGroups)
  int tile_npw = 4;       // node-group kernel: nodes per consumer warp (4: a warp per group; 2: two per group)
  int tile_rows = 1;      // node-group kernel: grid rows a tile spans (1..3)
  // fields of this many levels or fewer run on the per-node kernel unless
  // the node-group kernel is forced (group 2): its table work per tile does
  // not shrink with the levels.  Measured on O640 with union groups (node
  // group against per node, ms): FP32 gradient 30 levels 0.31 / 0.15, 60
  // levels 0.34 / 0.26, 91 levels 0.38 / 0.39; FP32 divergence 91 levels
  // 0.42 / 0.48; BF16 gradient 91 levels 0.39 / 0.34.  So 80 for FP32, 96
  // for BF16.  The Laplacian's per-node kernel is slower at any level
  // count, so its threshold is 0.
  int tile_min_levels = 96;
};

// Launch shape an fvm starts with, per operator and storage dtype: the
// autotuner's choice on O1280 x 137 on a GB300 (the tuner re-measures it on
// the caller's fields).  Two-ring Laplacian: 2 blocks of 512 threads per SM
// keep fewer neighbourhoods in L1; one-ring FP32: 256 threads, 3 entries per
// batch; bfloat16: tiles of 64 passes for the Laplacian.
LaunchCfg default_launch(int op, int dt) {
  LaunchCfg c;
  if (op == atlasgb::OP_LAP) c.tile_min_levels = 0;
  c.batch = 3;
  c.threads = 256;
  if (dt == ATLAS_F32) {
    if (op != atlasgb::OP_LAP) c.tile_min_levels = 80;
    // the node-group kernels: tiles of ten groups spanning two grid rows
    // (five groups of each), so the rows above and below are staged once
    // for both; one block per SM, union groups.  O1280 x 137: gradient 1.87
    // ms (1.90 with one-row tiles of eleven groups), divergence 2.19 (2.50
    // with one-row tiles of seven), Laplacian 2.31 (2.38 with two blocks
    // per SM of one-row tiles of four, 3.12 with per-node rows and two
    // warps per group)
    c.tile_groups = 10;
    c.tile_rows = 2;
    if (op == atlasgb::OP_LAP) {
      c.batch = 6;
      c.threads = 512;
      // the Laplacian's kernel needs fewer than 128 registers, so sixteen
      // warps fit and its tiles take twelve groups (six of each row):
      // 2.10 ms against 2.36 with ten
      c.tile_groups = 12;
    }
    if (op == atlasgb::OP_DIV_ADJ || op == atlasgb::OP_VGRAD) c.threads = 128;
  } else if (dt == ATLAS_BF16) {
    c.threads = 128;
    if (op == atlasgb::OP_LAP) c.tile_passes = 64;
    // bfloat16: tiles of eleven groups (their stages fit at half the
    // bytes), union groups; O1280 x 137: gradient 1.79 ms against 2.02 per
    // node, divergence 2.17 against 2.38.  The Laplacian takes fifteen
    // groups (sixteen warps under 128 registers): 2.15 ms against 2.43
    // with eleven and 4.38 per node.  The one-input operators' kernels fit
    // in 128 registers in bfloat16 too and take fifteen groups as well
    const bool one_in = op == atlasgb::OP_GRAD || op == atlasgb::OP_DIV_ADJ || op == atlasgb::OP_VGRAD ||
                        op == atlasgb::OP_CURL_ADJ;
    c.tile_groups = (op == atlasgb::OP_LAP || one_in) ? 15 : 11;
  } else {  // F64: bound by the FP64 pipe
    c.threads = 128;
  }
  return c;
}
}  // namespace

struct atlas_fvm_s {
  atlas_mesh_s* mesh = nullptr;
  atlasgb::Dual d;
  int device = -1;
  int num_sms = 0;
  std::mutex mu;
  OpTables st[atlasgb::OP_COUNT][3];  // [op][storage dtype: F32, F64, BF16]
  EdgeTables eg[3][2];                // [gradient, divergence, averaged-form gradient][precision]
  LaunchCfg cfg[atlasgb::OP_COUNT][3];  // [op][storage dtype], defaults from default_launch
  DevAlloc vmem;                       // FP64 dual volumes on the device (integrals)
  const double* d_V = nullptr;
  int users = 0;
};

namespace {

// ---------------------------------------------------------------- helpers
int elem_size(atlas_dtype t) { return t == ATLAS_F64 ? 8 : (t == ATLAS_BF16 ? 2 : 4); }
int prec_of(atlas_dtype t) { return t == ATLAS_F64 ? 1 : 0; }
StorageType storage_of(atlas_dtype t) {
  return t == ATLAS_F64 ? atlasgb::ST_F64 : (t == ATLAS_BF16 ? atlasgb::ST_BF16 : atlasgb::ST_F32);
}
bool valid_dtype(int t) { return t == ATLAS_F32 || t == ATLAS_F64 || t == ATLAS_BF16; }

int check_device(atlas_fvm_s* f) {
  if (f->device < 0) return fail(ATLAS_ECUDA, "no CUDA device was available when this fvm was built");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != f->device) return fail(ATLAS_ESTATE, "fvm lives on device %d, current device is %d", f->device, cur);
  return ATLAS_OK;
}


// Testing hook (atlas_debug_tile_hang): the next tile-kernel launches make
// their consumers wait on a barrier that nothing completes, with a short
// limit, so that the time-out path runs (no GPU fault, no hang).
std::atomic<int> g_tile_hang{0};
// Tuning hook (atlas_debug_tile_wait_hint): suspension hint of the
// consumers' barrier waits in nanoseconds, 0 for none.
std::atomic<unsigned> g_tile_wait_hint{0};
// Tuning hook (atlas_debug_tile_unions): 0 keeps every group in per-node
// form (tables built afterwards).
std::atomic<int> g_tile_unions{1};

// Tables for launches with nodes_per_warp npw carry union groups when every
// group has one warp.
bool wants_unions(int npw) { return npw == 4 && g_tile_unions.load() != 0; }


// Build and upload the tile tables of a stencil for float weights.  A
// stencil the tile layout cannot take leaves them absent (not an error);
// allocation failures are errors.
int build_group_tables(atlas_fvm_s* f, const atlasgb::Stencil& s, OpTables& t, int groups, bool unions, int rows) {
  GroupTables& g = t.grp;
  atlasgb::GroupStencil gs;
  atlasgb::TileStencil ts;
  try {
    if (!atlasgb::build_group_stencil(s, f->mesh->grid->g, gs)) return ATLAS_OK;
    if (!atlasgb::build_tile_stencil(gs, s, groups, ts, unions, rows)) return ATLAS_OK;
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building operator tables");
  }
  const int64_t nt = ts.ntiles;
  if (nt >= INT32_MAX) return ATLAS_OK;
  cudaError_t err = cudaSuccess;
  g.dev.head = g.mem.upload(ts.head, err);
  if (err == cudaSuccess) g.dev.blob = g.mem.upload(ts.blob, err);
  if (err != cudaSuccess) {
    g.mem.release();
    g.dev = atlasgb::DevTiles{};
    return err == cudaErrorMemoryAllocation ? fail(ATLAS_ENOMEM, "device allocation failed for operator tables")
                                            : cuda_fail(err, "upload of operator tables");
  }
  g.dev.ntiles = static_cast<int32_t>(nt);
  g.dev.max_slots = ts.max_slots;
  g.dev.max_blob = ts.max_blob;
  g.dev.blob_words = static_cast<int64_t>(ts.blob.size());
  g.dev.groups_per_tile = groups;
  g.dev.max_groups = ts.max_groups;
  g.dev.nin = s.nin;
  g.dev.nout = s.nout;
  g.dev.nw = ts.nw;
  g.dev.has_b = s.has_b;
  g.dev.unions = ts.unions;
  g.dev.union_groups = ts.union_groups;
  g.first.swap(ts.first);
  g.unit_tile.swap(ts.unit_tile);
  g.groups = groups;
  g.rows = rows;
  g.unions = unions;
  g.ok = true;
  return ATLAS_OK;
}

// Build and upload the stencil tables of op for fields of one storage dtype
// (double weights for F64 fields, float weights otherwise).
int ensure_stencil(atlas_fvm_s* f, int op, int dtype) {
  OpTables& t = f->st[op][dtype];
  const int prec = (dtype == ATLAS_F64) ? 1 : 0;
  if (t.ready) return ATLAS_OK;
  atlasgb::Stencil s;
  try {
    if (!atlasgb::build_stencil(f->mesh->m, f->d, op, s)) return fail(ATLAS_EINVAL, "stencil table overflow");
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building operator tables");
  }
  cudaError_t err = cudaSuccess;
  const int64_t V = f->mesh->grid->g.nnodes;
  t.dev.ptr = t.mem.upload(s.ptr, err);
  const size_t nnz = s.nbr.size();
  if (prec || s.nin == 2) {
    // double weights, or two-input operators: separate neighbour and weight arrays
    if (err == cudaSuccess) t.dev.nbr = t.mem.upload(s.nbr, err);
    std::vector<double> w = s.w;
    if (s.scalar_w) {
      std::vector<double> ws(nnz);
      for (size_t q = 0; q < nnz; ++q) ws[q] = s.w[2 * q];
      w.swap(ws);
    }
    if (err == cudaSuccess)
      t.dev.w = prec ? static_cast<const void*>(t.mem.upload(w, err))
                     : static_cast<const void*>(t.mem.upload(convert<float>(w), err));
  } else {
    // one-input operators, float weights: one packed entry per CSR slot,
    // {j, w} or {j, w0, w1, 0}
    const size_t stride = s.scalar_w ? 2 : 4;
    std::vector<uint32_t> ent(nnz * stride, 0u);
    for (size_t q = 0; q < nnz; ++q) {
      ent[stride * q] = static_cast<uint32_t>(s.nbr[q]);
      float w0 = static_cast<float>(s.w[2 * q]), w1 = static_cast<float>(s.w[2 * q + 1]);
      std::memcpy(&ent[stride * q + 1], &w0, 4);
      if (!s.scalar_w) std::memcpy(&ent[stride * q + 2], &w1, 4);
    }
    if (err == cudaSuccess) t.dev.w = t.mem.upload(ent, err);
  }
  if (err == cudaSuccess && s.has_b)
    t.dev.b = prec ? static_cast<const void*>(t.mem.upload(s.b, err))
                   : static_cast<const void*>(t.mem.upload(convert<float>(s.b), err));
  if (err != cudaSuccess) {
    t.mem.release();
    return err == cudaErrorMemoryAllocation ? fail(ATLAS_ENOMEM, "device allocation failed for operator tables")
                                            : cuda_fail(err, "upload of operator tables");
  }
  t.dev.nnodes = static_cast<int32_t>(V);
  t.dev.nnz = static_cast<int64_t>(s.nbr.size());
  t.dev.nin = s.nin;
  t.dev.nout = s.nout;
  t.dev.has_b = s.has_b;
  t.dev.scalar_w = s.scalar_w;
  if (!prec) {
    const LaunchCfg& c = f->cfg[op][dtype];
    const int rc = build_group_tables(f, s, t, c.tile_groups, wants_unions(c.tile_npw), c.tile_rows);
    if (rc) {
      t.mem.release();
      t.dev = atlasgb::DevStencil{};
      return rc;
    }
  }
  t.ready = true;
  return ATLAS_OK;
}

// Rebuild the tile tables when the groups per tile or the nodes per warp
// asked for with atlas_fvm_set_group differ from those built (caller holds
// the fvm lock; the stencil tables exist).  Tiles of one warp per group
// carry union groups, tiles of two warps per group do not.
int ensure_tile_layout(atlas_fvm_s* f, int op, int dtype) {
  OpTables& t = f->st[op][dtype];
  const int want = f->cfg[op][dtype].tile_groups, rows = f->cfg[op][dtype].tile_rows;
  const bool unions = wants_unions(f->cfg[op][dtype].tile_npw);
  if (dtype == ATLAS_F64 || !t.grp.ok || (t.grp.groups == want && t.grp.unions == unions && t.grp.rows == rows))
    return ATLAS_OK;
  atlasgb::Stencil s;
  try {
    if (!atlasgb::build_stencil(f->mesh->m, f->d, op, s)) return fail(ATLAS_EINVAL, "stencil table overflow");
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building operator tables");
  }
  // the per-node FP32 B term the tile tables point at stays in t.mem
  t.grp.mem.release();
  t.grp = GroupTables{};
  return build_group_tables(f, s, t, want, unions, rows);
}

int ensure_edges(atlas_fvm_s* f, int which /*0 grad, 1 div, 2 averaged-form grad*/, int prec) {
  EdgeTables& t = f->eg[which][prec];
  if (t.ready) return ATLAS_OK;
  const atlasgb::Mesh& m = f->mesh->m;
  if (f->mesh->grid->g.regional())
    return fail(ATLAS_EINVAL, "the edge-based two-pass variant covers global grids only");
  atlasgb::EdgeGather g;
  try {
    if (!atlasgb::build_edge_gather(m, f->d, which == 1 ? atlasgb::OP_DIV : atlasgb::OP_GRAD, g, which == 2))
      return fail(ATLAS_EINVAL, "edge table build failed");
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building edge tables");
  }
  const int64_t E = m.nedges, V = f->mesh->grid->g.nnodes;
  std::vector<double> coef(static_cast<size_t>(3 * E), 0.0), node(static_cast<size_t>(3 * V), 0.0);
  for (int64_t e = 0; e < E; ++e) {
    const double s0 = f->d.S[2 * e], s1 = f->d.S[2 * e + 1];
    if (which != 1) {
      coef[3 * e] = 0.5 * s0;
      coef[3 * e + 1] = 0.5 * s1;
    } else if (!m.is_pole[e]) {
      coef[3 * e] = 0.5 * s0;
      coef[3 * e + 1] = 0.5 * s1 * f->d.coslat[m.e2n[2 * e + 1]];
      coef[3 * e + 2] = 0.5 * s1 * g.dcos[e];
    }
  }
  for (int64_t i = 0; i < V; ++i) {
    node[3 * i] = g.inv_v[i];
    node[3 * i + 1] = which != 1 ? g.cos_v[i] : 0.0;
    node[3 * i + 2] = which != 1 ? 0.0 : g.pole_coef[i];
  }
  cudaError_t err = cudaSuccess;
  t.dev.e2n = t.mem.upload(m.e2n, err);
  if (err == cudaSuccess) t.dev.ptr = t.mem.upload(g.ptr, err);
  if (err == cudaSuccess) t.dev.ent = t.mem.upload(g.ent, err);
  if (err == cudaSuccess)
    t.dev.coef = prec ? static_cast<const void*>(t.mem.upload(coef, err))
                      : static_cast<const void*>(t.mem.upload(convert<float>(coef), err));
  if (err == cudaSuccess)
    t.dev.node = prec ? static_cast<const void*>(t.mem.upload(node, err))
                      : static_cast<const void*>(t.mem.upload(convert<float>(node), err));
  if (err != cudaSuccess) {
    t.mem.release();
    return err == cudaErrorMemoryAllocation ? fail(ATLAS_ENOMEM, "device allocation failed for edge tables")
                                            : cuda_fail(err, "upload of edge tables");
  }
  t.dev.nnodes = static_cast<int32_t>(V);
  t.dev.nedges = E;
  t.dev.nent = static_cast<int64_t>(g.ent.size());
  t.ready = true;
  return ATLAS_OK;
}

// Widest levels-per-thread vector that the dtype, ld and every pointer allow
// (capped by the requested width, 0 = no cap).
int pick_vec(atlas_dtype dt, int64_t ld, const void* const* ptrs, int nptr, int want) {
  const int es = elem_size(dt);
  int v = 16 / es;
  if (want > 0) v = std::min(v, want);
  while (v > 1) {
    bool okv = (ld % v) == 0;
    for (int k = 0; k < nptr && okv; ++k)
      if (ptrs[k] && (reinterpret_cast<uintptr_t>(ptrs[k]) % static_cast<uintptr_t>(v * es)) != 0) okv = false;
    if (okv) break;
    v >>= 1;
  }
  return v;
}

// Largest leading dimension: with fewer than 2^29 nodes in any grid and at
// most 8-byte elements, node * ld * element size then stays below 2^63.
constexpr int64_t kMaxLd = INT32_MAX;

int check_field_args(atlas_dtype dtype, int nlev, int64_t ld, const void* const* ptrs, int nptr) {
  if (!valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "unsupported dtype %d", static_cast<int>(dtype));
  if (nlev < 0) return fail(ATLAS_EINVAL, "nlev must be >= 0 (got %d)", nlev);
  if (ld < nlev || ld < 1) return fail(ATLAS_EINVAL, "leading dimension ld=%lld must be >= max(nlev, 1) (nlev=%d)",
                                       static_cast<long long>(ld), nlev);
  if (ld > kMaxLd)
    return fail(ATLAS_EINVAL, "leading dimension ld=%lld above 2^31 - 1", static_cast<long long>(ld));
  for (int k = 0; k < nptr; ++k) {
    if (!ptrs[k]) return fail(ATLAS_EINVAL, "field pointer %d is NULL", k);
    if (reinterpret_cast<uintptr_t>(ptrs[k]) % static_cast<uintptr_t>(elem_size(dtype)) != 0)
      return fail(ATLAS_EALIGN, "field pointer %d is not aligned to its element size", k);
  }
  return ATLAS_OK;
}

int check_no_overlap(const void* const* ins, int nin, void* const* outs, int nout, int64_t bytes) {
  auto overlaps = [bytes](const void* a, const void* b) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + static_cast<uintptr_t>(bytes) && y < x + static_cast<uintptr_t>(bytes);
  };
  for (int o = 0; o < nout; ++o) {
    for (int i = 0; i < nin; ++i)
      if (overlaps(outs[o], ins[i])) return fail(ATLAS_EINVAL, "output field %d overlaps input field %d", o, i);
    for (int p = o + 1; p < nout; ++p)
      if (overlaps(outs[o], outs[p])) return fail(ATLAS_EINVAL, "output fields %d and %d overlap", o, p);
  }
  return ATLAS_OK;
}

// As check_no_overlap, for inputs and outputs of different sizes.
int check_no_overlap2(const void* const* ins, int nin, int64_t in_bytes, void* const* outs, int nout,
                      int64_t out_bytes) {
  auto overlaps = [](const void* a, int64_t na, const void* b, int64_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + static_cast<uintptr_t>(nb) && y < x + static_cast<uintptr_t>(na);
  };
  for (int o = 0; o < nout; ++o) {
    for (int i = 0; i < nin; ++i)
      if (overlaps(outs[o], out_bytes, ins[i], in_bytes))
        return fail(ATLAS_EINVAL, "output field %d overlaps input field %d", o, i);
    for (int p = o + 1; p < nout; ++p)
      if (overlaps(outs[o], out_bytes, outs[p], out_bytes))
        return fail(ATLAS_EINVAL, "output fields %d and %d overlap", o, p);
  }
  return ATLAS_OK;
}

int grid_blocks(atlas_fvm_s* f, StorageType st, const atlasgb::DevStencil& s, int vec, int batch, int threads,
                int bps_req, int64_t items) {
  int bps = atlasgb::stencil_occupancy(st, s, vec, batch, threads);
  if (bps_req > 0) bps = std::min(bps, bps_req);
  int64_t blocks = static_cast<int64_t>(f->num_sms) * bps;
  const int64_t need = (items + threads - 1) / threads;
  if (need < blocks) blocks = need;
  return static_cast<int>(std::max<int64_t>(blocks, 1));
}

atlas_fvm_s* get_fvm(atlas_fvm_t h) { return live(h) ? reinterpret_cast<atlas_fvm_s*>(h) : nullptr; }

// Level layout of the node-group kernels: part A holds va levels per lane
// (32 va per level block), part B vb; the narrowest pair whose block covers
// nlev levels, within the vector width the rows' alignment allows (vmax).
void group_layout(int nlev, int vmax, int& va, int& vb) {
  if (vmax >= 4) {
    if (nlev <= 32) { va = 1; vb = 0; }
    else if (nlev <= 64) { va = 2; vb = 0; }
    else if (nlev <= 96) { va = 2; vb = 1; }
    else if (nlev <= 128) { va = 4; vb = 0; }
    else if (nlev <= 160) { va = 4; vb = 1; }
    else { va = 4; vb = 2; }
  } else if (vmax >= 2) {
    if (nlev <= 32) { va = 1; vb = 0; }
    else if (nlev <= 64) { va = 2; vb = 0; }
    else { va = 2; vb = 1; }
  } else {
    va = 1;
    vb = 0;
  }
}

// Launch of the shared-memory node-group kernel over tiles [t0, t0 + nt)
// with pointers already shifted to global node ids (see run_stencil_range).
int run_tiles(atlas_fvm_s* f, const GroupTables& gt, const LaunchCfg& c, StorageType st, const void* in0,
              const void* in1, void* out0, void* out1, int nlev, int64_t ld, atlas_dtype dtype,
              const void* const* used, int nu, int32_t t0, int32_t nt, atlasgb::Bounds bd, void* stream) {
  if (nt == 0) return ok();
  atlasgb::TileLaunch l;
  l.in0 = in0;
  l.in1 = in1;
  l.out0 = out0;
  l.out1 = out1;
  l.nlev = nlev;
  l.ld = ld;
  group_layout(nlev, pick_vec(dtype, ld, used, nu, 4), l.va, l.vb);
  // padding levels written as zeros: up to the end of the widest vector
  // the rows allow (the per-node kernels' rule)
  const int vpad = pick_vec(dtype, ld, used, nu, 0);
  l.nstore = static_cast<int32_t>(std::min<int64_t>(ld, (nlev + vpad - 1) / vpad * vpad));
  l.t0 = t0;
  l.ntiles = nt;
  l.bd = bd;
  l.sms = f->num_sms;
  l.max_bps = c.tile_bps;
  l.npw = gt.dev.unions ? 4 : c.tile_npw;  // union groups need a warp per group
  l.wait_hint_ns = g_tile_wait_hint.load();
  if (g_tile_hang.load()) {
    l.hang_test = 1;
    l.wait_limit = 1ll << 22;  // a few milliseconds
  }
  cudaError_t e = atlasgb::launch_tiles(st, gt.dev, l, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "node-group kernel launch");
  const int rc = bounds_after(stream, "node-group kernel");
  return rc ? rc : ok();
}

// One fused node-stencil operator over nodes [node0, node0 + count).  The
// input fields hold the nodes from in_first on (their row 0 is node
// in_first, in_nodes rows), the outputs the nodes from node0 on (count
// rows).  The kernels index fields by global node id: each pointer is
// shifted back by its first node (integer arithmetic on the address; the
// kernel only touches rows inside the buffer).
int run_stencil_range(atlas_fvm_s* f, int op, const void* in0, const void* in1, void* out0, void* out1, int nlev,
                      int64_t ld, atlas_dtype dtype, void* stream, int64_t node0, int64_t count, int64_t in_first,
                      int64_t in_nodes) {
  const void* ins[2] = {in0, in1};
  void* outs[2] = {out0, out1};
  const int nin = (op == atlasgb::OP_DIV || op == atlasgb::OP_GRAD_ADJ || op == atlasgb::OP_CURL) ? 2 : 1;
  const int nout =
      (op == atlasgb::OP_GRAD || op == atlasgb::OP_DIV_ADJ || op == atlasgb::OP_VGRAD || op == atlasgb::OP_CURL_ADJ) ? 2
                                                                                                                  : 1;
  const void* used[4];
  int nu = 0;
  for (int k = 0; k < nin; ++k) used[nu++] = ins[k];
  for (int k = 0; k < nout; ++k) used[nu++] = outs[k];
  int rc = check_field_args(dtype, nlev, ld, used, nu);
  if (rc) return rc;
  const int64_t es = elem_size(dtype);
  rc = check_no_overlap2(ins, nin, in_nodes * ld * es, outs, nout, count * ld * es);
  if (rc) return rc;
  rc = check_device(f);
  if (rc) return rc;
  if (nlev == 0 || count == 0) return ok();
  {
    std::lock_guard<std::mutex> lk(f->mu);
    rc = ensure_stencil(f, op, dtype);
    if (rc) return rc;
    rc = ensure_tile_layout(f, op, dtype);
    if (rc) return rc;
  }
  const atlasgb::DevStencil& dev = f->st[op][dtype].dev;
  const GroupTables& gt = f->st[op][dtype].grp;
  auto shift = [&](const void* p, int64_t first) -> const void* {
    return p ? reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(p) -
                                             static_cast<uintptr_t>(first * ld * es))
             : nullptr;
  };
  const LaunchCfg& c = f->cfg[op][dtype];
  const StorageType st = storage_of(dtype);
  atlasgb::Bounds bd;  // checked by the bounds-checked build's kernels
  bd.lo = static_cast<int32_t>(in_first);
  bd.hi = static_cast<int32_t>(in_first + in_nodes);
  bd.olo = static_cast<int32_t>(node0);
  bd.ohi = static_cast<int32_t>(node0 + count);
  bd.err = atlasgb::bounds_word();
  // the node-group kernel where it pays (LaunchCfg::tile_min_levels)
  const bool tiles_wanted = c.group == 2 || (c.group == 1 && nlev > c.tile_min_levels);
  // the per-node kernel over nodes [n0, n0 + cnt) of the range
  auto per_node = [&](int64_t n0, int64_t cnt) -> int {
    if (cnt == 0) return ATLAS_OK;
    atlasgb::StencilLaunch l;
    l.in0 = shift(in0, in_first);
    l.in1 = nin == 2 ? shift(in1, in_first) : nullptr;
    l.out0 = const_cast<void*>(shift(out0, node0));
    l.out1 = nout == 2 ? const_cast<void*>(shift(out1, node0)) : nullptr;
    l.nlev = nlev;
    l.ld = ld;
    l.node0 = static_cast<int32_t>(n0);
    l.count = static_cast<int32_t>(cnt);
    l.vec = pick_vec(dtype, ld, used, nu, c.vec);
    const int64_t nvec = (nlev + l.vec - 1) / l.vec;
    const int64_t items = cnt * nvec;
    if (f->mesh->grid->g.nnodes * nvec >= (int64_t(1) << 31))
      return fail(ATLAS_EINVAL, "nnodes * level-vectors must stay below 2^31");
    l.threads = c.threads;
    l.batch = c.batch;
    l.blocks = grid_blocks(f, st, dev, l.vec, l.batch, l.threads, c.blocks_per_sm, items);
    {
      // a tile is at most one block's even share, so blocks * tile stays
      // below 2^31 + blocks * threads
      const int64_t share = ((items + l.blocks - 1) / l.blocks + l.threads - 1) / l.threads * l.threads;
      l.tile = static_cast<uint32_t>(
          std::max<int64_t>(l.threads, std::min<int64_t>(int64_t(c.tile_passes) * l.threads, share)));
    }
    atlasgb::Bounds b2 = bd;
    b2.nnz = dev.nnz;
    l.bd = b2;
    cudaError_t e = atlasgb::launch_stencil(st, dev, l, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stencil kernel launch");
    return bounds_after(stream, "stencil kernel");
  };
  const int npw = gt.dev.unions ? 4 : c.tile_npw;  // as run_tiles launches
  const bool tiles_fit =
      gt.ok && 32 * ((4 / npw) * gt.dev.max_groups + 1) <=
                   atlasgb::tile_max_threads(npw, gt.dev.nin, gt.dev.nout, static_cast<int>(es));
  if (gt.ok && tiles_wanted && tiles_fit && (ld * es) % 16 == 0 &&
      atlasgb::tile_smem_bytes(gt.dev, ld, static_cast<int>(es)) > 0) {
    // the shared-memory node-group kernel: TMA copies need 16-byte aligned
    // rows; it takes the whole units (runs of grid rows whose tiles are
    // consecutive) inside the range, the per-node kernel the rest (the
    // rows of units the range cuts), with identical results
    bool aligned = true;
    for (int k = 0; k < nu; ++k)
      if (reinterpret_cast<uintptr_t>(used[k]) % 16 != 0) aligned = false;
    const auto a = std::lower_bound(gt.first.begin(), gt.first.end(), node0);
    auto b = std::upper_bound(gt.first.begin(), gt.first.end(), node0 + count);
    if (b != gt.first.begin()) --b;
    if (aligned && a != gt.first.end() && a < b) {
      const int32_t t0 = gt.unit_tile[static_cast<size_t>(a - gt.first.begin())];
      const int32_t t1 = gt.unit_tile[static_cast<size_t>(b - gt.first.begin())];
      rc = run_tiles(f, gt, c, st, shift(in0, in_first), nin == 2 ? shift(in1, in_first) : nullptr,
                     const_cast<void*>(shift(out0, node0)), nout == 2 ? const_cast<void*>(shift(out1, node0)) : nullptr,
                     nlev, ld, dtype, used, nu, t0, t1 - t0, bd, stream);
      if (rc) return rc;
      rc = per_node(node0, *a - node0);
      if (rc) return rc;
      rc = per_node(*b, node0 + count - *b);
      return rc ? rc : ok();
    }
  }
  rc = per_node(node0, count);
  return rc ? rc : ok();
}

// The operator over every node, on whole fields.
int run_stencil_op(atlas_fvm_t h, int op, const void* in0, const void* in1, void* out0, void* out1, int nlev,
                   int64_t ld, atlas_dtype dtype, void* stream) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  const int64_t V = f->mesh->grid->g.nnodes;
  return run_stencil_range(f, op, in0, in1, out0, out1, nlev, ld, dtype, stream, 0, V, 0, V);
}

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

struct WsLayout {
  size_t flux0 = 0, flux1 = 0, g0 = 0, g1 = 0, total = 0;
};
WsLayout ws_layout(atlas_fvm_s* f, int op, int64_t ld, atlas_dtype dt) {
  WsLayout w;
  const int64_t E = f->mesh->m.nedges, V = f->mesh->grid->g.nnodes;
  const size_t ab = dt == ATLAS_F64 ? 8 : 4;
  const size_t fbytes = align256(static_cast<size_t>(E) * ld * ab);
  const size_t gbytes = align256(static_cast<size_t>(V) * ld * elem_size(dt));
  size_t o = 0;
  w.flux0 = o;
  o += fbytes;
  if (op == ATLAS_OP_GRADIENT || op == ATLAS_OP_LAPLACIAN) {
    w.flux1 = o;
    o += fbytes;
  }
  if (op == ATLAS_OP_LAPLACIAN) {
    w.g0 = o;
    o += gbytes;
    w.g1 = o;
    o += gbytes;
  }
  w.total = o;
  return w;
}

int edge_blocks(atlas_fvm_s* f, int64_t items, int threads) {
  int64_t blocks = static_cast<int64_t>(f->num_sms) * 8;
  const int64_t need = (items + threads - 1) / threads;
  return static_cast<int>(std::max<int64_t>(1, std::min(blocks, need)));
}

// Edge-based two-kernel gradient (which = 0) or divergence (which = 1).
int run_edges_op(atlas_fvm_s* f, int which, const void* in0, const void* in1, void* out0, void* out1, char* ws,
                 const WsLayout& w, int nlev, int64_t ld, atlas_dtype dtype, cudaStream_t stream, int vec_cap = 0) {
  const int prec = prec_of(dtype);
  {
    std::lock_guard<std::mutex> lk(f->mu);
    int rc = ensure_edges(f, which, prec);
    if (rc) return rc;
  }
  const atlasgb::DevEdges& E = f->eg[which][prec].dev;
  const void* ptrs[5] = {in0, in1, out0, out1, ws};
  const int cap = f->cfg[which == 1 ? 1 : 0][dtype].vec;
  const int vec = pick_vec(dtype, ld, ptrs, 5, vec_cap > 0 ? (cap > 0 ? std::min(cap, vec_cap) : vec_cap) : cap);
  const int64_t nvec = (nlev + vec - 1) / vec;
  if (E.nedges * nvec >= (int64_t(1) << 31)) return fail(ATLAS_EINVAL, "nedges * level-vectors must stay below 2^31");
  const int threads = 256;
  const StorageType st = storage_of(dtype);
  const bool grad = which != 1;
  cudaError_t e = atlasgb::launch_edge_flux(st, which, E, in0, in1, ws + w.flux0, grad ? ws + w.flux1 : nullptr,
                                            nlev, ld, vec, threads, edge_blocks(f, E.nedges * nvec, threads), stream);
  if (e != cudaSuccess) return cuda_fail(e, "edge-flux kernel launch");
  e = atlasgb::launch_node_gather(st, grad ? 0 : 1, E, ws + w.flux0, grad ? ws + w.flux1 : nullptr,
                                  which == 1 ? in1 : nullptr, out0, grad ? out1 : nullptr, nlev, ld, vec, threads,
                                  edge_blocks(f, static_cast<int64_t>(E.nnodes) * nvec, threads), stream);
  if (e != cudaSuccess) return cuda_fail(e, "node-gather kernel launch");
  return bounds_after(stream, "edge-flux and node-gather kernels");
}

int check_ws(atlas_fvm_s* f, int op, void* ws, size_t ws_bytes, int64_t ld, atlas_dtype dt, WsLayout& w) {
  w = ws_layout(f, op, ld, dt);
  if (!ws) return fail(ATLAS_EINVAL, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(ATLAS_EALIGN, "workspace must be 256-byte aligned");
  if (ws_bytes < w.total)
    return fail(ATLAS_EINVAL, "workspace too small: %zu bytes given, %zu needed", ws_bytes, w.total);
  return ATLAS_OK;
}

const char* kVersion = "atlasgb 0.1.0 (sm_103a)";

}  // namespace

// =================================================================== C ABI
extern "C" {

int atlas_init(void) { return ok(); }
int atlas_finalize(void) { return ok(); }
const char* atlas_version(void) { return kVersion; }

const char* atlas_info(void) {
  static thread_local std::string s;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  char buf[512];
  if (e != cudaSuccess || n == 0) {
    std::snprintf(buf, sizeof buf, "%s%s; no CUDA device (%s)", kVersion,
                  atlasgb::bounds_checked() ? " (bounds-checked kernels)" : "", cudaGetErrorString(e));
  } else {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, dev);
    std::snprintf(buf, sizeof buf, "%s%s; device %d: %s, sm_%d%d, %d SMs, %.1f GiB", kVersion,
                  atlasgb::bounds_checked() ? " (bounds-checked kernels)" : "", dev, p.name, p.major, p.minor,
                  p.multiProcessorCount, static_cast<double>(p.totalGlobalMem) / (1 << 30));
  }
  s = buf;
  return s.c_str();
}

const char* atlas_last_error(void) { return g_err.c_str(); }

int atlas_grid_octahedral(int N, atlas_grid_t* out) {
  CallRange range_("atlas_grid_octahedral");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (N < 1 || N > 8000) return fail(ATLAS_EINVAL, "octahedral number N=%d out of range [1, 8000]", N);
  atlas_grid_s* g = new (std::nothrow) atlas_grid_s();
  if (!g) return fail(ATLAS_ENOMEM, "out of host memory");
  try {
    if (!atlasgb::build_grid(N, g->g)) {
      delete g;
      return fail(ATLAS_EINVAL, "grid build failed");
    }
  } catch (const std::bad_alloc&) {
    delete g;
    return fail(ATLAS_ENOMEM, "out of host memory building O%d", N);
  }
  reg(g);
  *out = reinterpret_cast<atlas_grid_t>(g);
  return ok();
}

int atlas_grid_regular_gaussian(int N, atlas_grid_t* out) {
  CallRange range_("atlas_grid_regular_gaussian");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (N < 1 || N > 8000) return fail(ATLAS_EINVAL, "Gaussian number N=%d out of range [1, 8000]", N);
  atlas_grid_s* g = new (std::nothrow) atlas_grid_s();
  if (!g) return fail(ATLAS_ENOMEM, "out of host memory");
  try {
    if (!atlasgb::build_regular_gaussian_grid(N, g->g)) {
      delete g;
      return fail(ATLAS_EINVAL, "grid build failed");
    }
  } catch (const std::bad_alloc&) {
    delete g;
    return fail(ATLAS_ENOMEM, "out of host memory building F%d", N);
  }
  reg(g);
  *out = reinterpret_cast<atlas_grid_t>(g);
  return ok();
}

int atlas_grid_regional(int projection, int nx, int ny, const double* params, atlas_grid_t* out) {
  CallRange range_("atlas_grid_regional");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (projection < ATLAS_PROJ_ROTATED_LONLAT || projection > ATLAS_PROJ_POLAR_STEREOGRAPHIC)
    return fail(ATLAS_EINVAL, "unknown projection %d", projection);
  atlas_grid_s* g = new (std::nothrow) atlas_grid_s();
  if (!g) return fail(ATLAS_ENOMEM, "out of host memory");
  const char* why = "invalid regional grid";
  try {
    if (!atlasgb::build_regional_grid(projection, nx, ny, params, g->g, &why)) {
      delete g;
      return fail(ATLAS_EINVAL, "%s", why);
    }
  } catch (const std::bad_alloc&) {
    delete g;
    return fail(ATLAS_ENOMEM, "out of host memory building a %d x %d regional grid", nx, ny);
  }
  reg(g);
  *out = reinterpret_cast<atlas_grid_t>(g);
  return ok();
}

int atlas_grid_regional_info(atlas_grid_t h, int* projection, int* nx, int* ny, const double** xy,
                             const double** scale) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed grid handle");
  const atlasgb::Grid& g = reinterpret_cast<atlas_grid_s*>(h)->g;
  if (!g.regional()) return fail(ATLAS_EINVAL, "not a regional grid");
  if (projection) *projection = g.projection;
  if (nx) *nx = g.nx;
  if (ny) *ny = g.nlat;
  if (xy) *xy = g.xy.data();
  if (scale) *scale = g.h.data();
  return ok();
}

int atlas_grid_info(atlas_grid_t h, int64_t* nnodes, int* nlat, const int32_t** pl, const double** lonlat,
                    const double** lat) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed grid handle");
  const atlasgb::Grid& g = reinterpret_cast<atlas_grid_s*>(h)->g;
  if (nnodes) *nnodes = g.nnodes;
  if (nlat) *nlat = g.nlat;
  if (pl) *pl = g.pl.data();
  if (lonlat) *lonlat = g.lonlat.data();
  if (lat) *lat = g.lat.data();
  return ok();
}

void atlas_grid_destroy(atlas_grid_t h) {
  if (!live(h)) return;
  atlas_grid_s* g = reinterpret_cast<atlas_grid_s*>(h);
  if (g->users > 0) {
    fail(ATLAS_ESTATE, "grid still used by %d mesh(es) or remap(s); not destroyed", g->users);
    return;
  }
  unreg(g);
  delete g;
}

int atlas_mesh_build(atlas_grid_t gh, atlas_mesh_t* out) {
  CallRange range_("atlas_mesh_build");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!live(gh)) return fail(ATLAS_ESTATE, "invalid or destroyed grid handle");
  atlas_grid_s* g = reinterpret_cast<atlas_grid_s*>(gh);
  atlas_mesh_s* m = new (std::nothrow) atlas_mesh_s();
  if (!m) return fail(ATLAS_ENOMEM, "out of host memory");
  try {
    if (!atlasgb::build_mesh(g->g, m->m)) {
      delete m;
      return fail(ATLAS_EINVAL, "mesh build failed (inconsistent zipper)");
    }
  } catch (const std::bad_alloc&) {
    delete m;
    return fail(ATLAS_ENOMEM, "out of host memory building the mesh");
  }
  m->grid = g;
  g->users++;
  reg(m);
  *out = reinterpret_cast<atlas_mesh_t>(m);
  return ok();
}

int atlas_mesh_info(atlas_mesh_t h, int64_t* nedges, int64_t* ntri, const int32_t** e2n, const uint8_t** is_pole,
                    const int32_t** n2e_ptr, const int32_t** n2e, const int8_t** n2e_sign, const int32_t** tri) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed mesh handle");
  const atlasgb::Mesh& m = reinterpret_cast<atlas_mesh_s*>(h)->m;
  if (nedges) *nedges = m.nedges;
  if (ntri) *ntri = m.ntri;
  if (e2n) *e2n = m.e2n.data();
  if (is_pole) *is_pole = m.is_pole.data();
  if (n2e_ptr) *n2e_ptr = m.n2e_ptr.data();
  if (n2e) *n2e = m.n2e.data();
  if (n2e_sign) *n2e_sign = m.n2e_sign.data();
  if (tri) *tri = m.tri.data();
  return ok();
}

void atlas_mesh_destroy(atlas_mesh_t h) {
  if (!live(h)) return;
  atlas_mesh_s* m = reinterpret_cast<atlas_mesh_s*>(h);
  if (m->users > 0) {
    fail(ATLAS_ESTATE, "mesh still used by %d fvm(s) or remap(s); not destroyed", m->users);
    return;
  }
  unreg(m);
  m->grid->users--;
  delete m;
}

int atlas_fvm_build_dual(atlas_mesh_t mh, double radius, atlas_fvm_t* out) {
  CallRange range_("atlas_fvm_build_dual");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!live(mh)) return fail(ATLAS_ESTATE, "invalid or destroyed mesh handle");
  if (!(radius > 0) || radius > 1e12) return fail(ATLAS_EINVAL, "radius must be positive and finite");
  atlas_mesh_s* m = reinterpret_cast<atlas_mesh_s*>(mh);
  atlas_fvm_s* f = new (std::nothrow) atlas_fvm_s();
  if (!f) return fail(ATLAS_ENOMEM, "out of host memory");
  for (int op = 0; op < atlasgb::OP_COUNT; ++op)
    for (int dt = 0; dt < 3; ++dt) f->cfg[op][dt] = default_launch(op, dt);
  try {
    if (!atlasgb::build_dual(m->m, radius, f->d)) {
      delete f;
      return fail(ATLAS_EINVAL, "dual build failed");
    }
    double worst = 0.0;
    int64_t node = -1;
    const char* why = "";
    if (!atlasgb::check_geometry(m->m, f->d, 1e-12, worst, node, &why)) {
      delete f;
      return fail(ATLAS_EINVAL, "dual build gave an inconsistent geometry: %s (node %lld)", why,
                  static_cast<long long>(node));
    }
  } catch (const std::bad_alloc&) {
    delete f;
    return fail(ATLAS_ENOMEM, "out of host memory building the dual");
  }
  f->mesh = m;
  int n = 0;
  if (cudaGetDeviceCount(&n) == cudaSuccess && n > 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    f->device = dev;
    cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, dev);
  } else {
    cudaGetLastError();  // clear the sticky "no device" status of the runtime
    f->device = -1;
  }
  m->users++;
  reg(f);
  *out = reinterpret_cast<atlas_fvm_t>(f);
  return ok();
}

int atlas_fvm_info(atlas_fvm_t h, const double** V, const double** S, const double** coslat, const double** pole_nphi) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (V) *V = f->d.V.data();
  if (S) *S = f->d.S.data();
  if (coslat) *coslat = f->d.coslat.data();
  if (pole_nphi) *pole_nphi = f->d.pole_nphi.data();
  return ok();
}

int atlas_fvm_regional_info(atlas_fvm_t h, const double** area, const double** Sb) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (!f->mesh->grid->g.regional()) return fail(ATLAS_EINVAL, "not the dual of a regional grid");
  if (area) *area = f->d.A.data();
  if (Sb) *Sb = f->d.Sb.data();
  return ok();
}

int atlas_fvm_check(atlas_fvm_t h, double* worst_closure) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  double worst = 0.0;
  int64_t node = -1;
  const char* why = "inconsistent geometry";
  const bool good = atlasgb::check_geometry(f->mesh->m, f->d, 1e-12, worst, node, &why);
  if (worst_closure) *worst_closure = worst;
  if (!good) {
    if (node >= 0) return fail(ATLAS_EINVAL, "%s (node %lld)", why, static_cast<long long>(node));
    return fail(ATLAS_EINVAL, "%s", why);
  }
  return ok();
}

int atlas_fvm_radius(atlas_fvm_t h, double* radius) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (!radius) return fail(ATLAS_EINVAL, "radius is NULL");
  *radius = f->d.R;
  return ok();
}

int atlas_fvm_save(atlas_fvm_t h, const char* path) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (!path) return fail(ATLAS_EINVAL, "path is NULL");
  const char* why = "";
  try {
    if (!atlasgb::save_geometry(f->mesh->grid->g, f->mesh->m, f->d, path, &why))
      return fail(ATLAS_EINVAL, "saving the geometry to %s: %s", path, why);
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "out of host memory saving the geometry");
  }
  return ok();
}

int atlas_fvm_load(const char* path, atlas_grid_t* grid, atlas_mesh_t* mesh, atlas_fvm_t* out) {
  if (!path || !grid || !mesh || !out) return fail(ATLAS_EINVAL, "NULL argument");
  *grid = nullptr;
  *mesh = nullptr;
  *out = nullptr;
  atlas_grid_s* g = new (std::nothrow) atlas_grid_s();
  atlas_mesh_s* m = new (std::nothrow) atlas_mesh_s();
  atlas_fvm_s* f = new (std::nothrow) atlas_fvm_s();
  auto drop = [&]() {
    delete f;
    delete m;
    delete g;
  };
  if (!g || !m || !f) {
    drop();
    return fail(ATLAS_ENOMEM, "out of host memory");
  }
  const char* why = "";
  try {
    if (!atlasgb::load_geometry(path, g->g, m->m, f->d, &why)) {
      drop();
      return fail(ATLAS_EINVAL, "loading the geometry from %s: %s", path, why);
    }
    double worst = 0.0;
    int64_t node = -1;
    if (!atlasgb::check_geometry(m->m, f->d, 1e-12, worst, node, &why)) {
      drop();
      return fail(ATLAS_EINVAL, "the geometry in %s is inconsistent: %s (node %lld)", path, why,
                  static_cast<long long>(node));
    }
  } catch (const std::bad_alloc&) {
    drop();
    return fail(ATLAS_ENOMEM, "out of host memory loading the geometry");
  }
  for (int op = 0; op < atlasgb::OP_COUNT; ++op)
    for (int dt = 0; dt < 3; ++dt) f->cfg[op][dt] = default_launch(op, dt);
  m->grid = g;
  g->users++;
  f->mesh = m;
  m->users++;
  int n = 0;
  if (cudaGetDeviceCount(&n) == cudaSuccess && n > 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    f->device = dev;
    cudaDeviceGetAttribute(&f->num_sms, cudaDevAttrMultiProcessorCount, dev);
  } else {
    cudaGetLastError();
    f->device = -1;
  }
  reg(g);
  reg(m);
  reg(f);
  *grid = reinterpret_cast<atlas_grid_t>(g);
  *mesh = reinterpret_cast<atlas_mesh_t>(m);
  *out = reinterpret_cast<atlas_fvm_t>(f);
  return ok();
}

int atlas_debug_fail_allocations(int after) {
  if (after < -1) return fail(ATLAS_EINVAL, "after must be >= -1");
  g_alloc_budget.store(after);
  return ok();
}

int atlas_fvm_prepare(atlas_fvm_t h, unsigned op_mask, unsigned dtype_mask) {
  CallRange range_("atlas_fvm_prepare");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  int rc = check_device(f);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(f->mu);
  for (int op = 0; op < atlasgb::OP_COUNT; ++op) {
    if (!(op_mask & (1u << op))) continue;
    for (int dt = 0; dt < 3; ++dt) {
      if (!(dtype_mask & (1u << dt))) continue;
      rc = ensure_stencil(f, op, dt);
      if (rc) return rc;
      if (op <= atlasgb::OP_DIV && dt != ATLAS_BF16 && !f->mesh->grid->g.regional()) {
        rc = ensure_edges(f, op, prec_of(static_cast<atlas_dtype>(dt)));
        if (rc) return rc;
      }
    }
  }
  return ok();
}

int atlas_fvm_set_launch(atlas_fvm_t h, int op, int dtype, int vec, int batch, int threads, int blocks_per_sm,
                         int tile_passes) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (dtype != -1 && !valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "dtype must be -1 (all) or an atlas_dtype");
  if (vec != 0 && vec != 1 && vec != 2 && vec != 4 && vec != 8) return fail(ATLAS_EINVAL, "vec must be 1, 2, 4 or 8");
  if (batch != 0 && batch != 3 && batch != 6) return fail(ATLAS_EINVAL, "batch must be 3 or 6");
  if (threads != 0 && (threads < 64 || threads > 512 || threads % 32 != 0))
    return fail(ATLAS_EINVAL, "threads must be a multiple of 32 in [64, 512]");
  if (blocks_per_sm < 0 || blocks_per_sm > 32) return fail(ATLAS_EINVAL, "blocks_per_sm must be in [0, 32]");
  if (tile_passes < 0 || tile_passes > 4096) return fail(ATLAS_EINVAL, "tile_passes must be in [0, 4096]");
  std::lock_guard<std::mutex> lk(f->mu);
  for (int d = 0; d < 3; ++d) {
    if (dtype != -1 && d != dtype) continue;
    LaunchCfg& c = f->cfg[op][d];
    if (vec) c.vec = vec;
    if (batch) c.batch = batch;
    if (threads) c.threads = threads;
    if (blocks_per_sm) c.blocks_per_sm = blocks_per_sm;
    if (tile_passes) c.tile_passes = tile_passes;
  }
  return ok();
}

int atlas_fvm_set_group(atlas_fvm_t h, int op, int dtype, int enable, int blocks_per_sm, int groups_per_tile,
                        int nodes_per_warp, int rows_per_tile) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (dtype != -1 && !valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "dtype must be -1 (all) or an atlas_dtype");
  if (enable < -1 || enable > 2) return fail(ATLAS_EINVAL, "enable must be -1, 0, 1 or 2");
  if (blocks_per_sm < 0 || blocks_per_sm > 2) return fail(ATLAS_EINVAL, "blocks_per_sm must be 0, 1 or 2");
  if (groups_per_tile < 0 || groups_per_tile > atlasgb::kTileMaxGroups)
    return fail(ATLAS_EINVAL, "groups_per_tile must be in [0, %d]", atlasgb::kTileMaxGroups);
  if (nodes_per_warp != 0 && nodes_per_warp != 2 && nodes_per_warp != 4)
    return fail(ATLAS_EINVAL, "nodes_per_warp must be 0, 2 or 4");
  if (rows_per_tile < 0 || rows_per_tile > atlasgb::kMaxTileRows)
    return fail(ATLAS_EINVAL, "rows_per_tile must be in [0, %d]", atlasgb::kMaxTileRows);
  std::lock_guard<std::mutex> lk(f->mu);
  for (int d = 0; d < 3; ++d) {
    if (dtype != -1 && d != dtype) continue;
    if (enable >= 0) f->cfg[op][d].group = enable;
    if (blocks_per_sm) f->cfg[op][d].tile_bps = blocks_per_sm;
    if (groups_per_tile) f->cfg[op][d].tile_groups = groups_per_tile;
    if (nodes_per_warp) f->cfg[op][d].tile_npw = nodes_per_warp;
    if (rows_per_tile) f->cfg[op][d].tile_rows = rows_per_tile;
  }
  return ok();
}

int atlas_fvm_tile_info(atlas_fvm_t h, int op, int dtype, int nlev, int64_t ld, int* blocks_per_sm, int* stages,
                        int64_t* smem_bytes, int64_t* max_rows) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (!valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "unsupported dtype %d", dtype);
  if (nlev < 1 || ld < nlev) return fail(ATLAS_EINVAL, "need 1 <= nlev <= ld");
  int rc = check_device(f);
  if (rc) return rc;
  if (blocks_per_sm) *blocks_per_sm = 0;
  if (stages) *stages = 0;
  if (smem_bytes) *smem_bytes = 0;
  if (max_rows) *max_rows = 0;
  {
    std::lock_guard<std::mutex> lk(f->mu);
    rc = ensure_stencil(f, op, dtype);
    if (rc) return rc;
    rc = ensure_tile_layout(f, op, dtype);
    if (rc) return rc;
  }
  const GroupTables& gt = f->st[op][dtype].grp;
  const int es = elem_size(static_cast<atlas_dtype>(dtype));
  if (!gt.ok || (ld * es) % 16 != 0) return ok();
  atlasgb::TileLaunch l;
  l.nlev = nlev;
  l.ld = ld;
  const void* none[1] = {nullptr};
  group_layout(nlev, pick_vec(static_cast<atlas_dtype>(dtype), ld, none, 0, 4), l.va, l.vb);
  l.sms = f->num_sms;
  l.max_bps = f->cfg[op][dtype].tile_bps;
  l.npw = gt.dev.unions ? 4 : f->cfg[op][dtype].tile_npw;
  int b = 0, s = 0;
  size_t m = 0;
  cudaError_t e = atlasgb::tile_shape(storage_of(static_cast<atlas_dtype>(dtype)), gt.dev, l, &b, &s, &m);
  if (e != cudaSuccess) return cuda_fail(e, "tile launch shape");
  if (blocks_per_sm) *blocks_per_sm = b;
  if (stages) *stages = s;
  if (smem_bytes) *smem_bytes = static_cast<int64_t>(m);
  if (max_rows) *max_rows = gt.dev.max_slots;
  return ok();
}

int atlas_fp64_fma_rate_kernel(double* out, int blocks, int threads, int64_t iters, void* stream) {
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 != 0 || iters < 0)
    return fail(ATLAS_EINVAL, "need blocks >= 1, threads a multiple of 32 in [32, 256], iters >= 0");
  if (reinterpret_cast<uintptr_t>(out) % 8 != 0) return fail(ATLAS_EALIGN, "out must be 8-byte aligned");
  cudaError_t e = atlasgb::launch_fp64_fma(out, blocks, threads, iters, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "FP64 rate kernel launch");
  return ok();
}

int atlas_kernel_status(unsigned* code, int clear) {
  if (!code) return fail(ATLAS_EINVAL, "code is NULL");
  *code = 0;
  cudaError_t e = atlasgb::tile_error(code, clear != 0);
  if (e != cudaSuccess) return cuda_fail(e, "reading the kernels' error word");
  return ok();
}

int atlas_debug_tile_wait_hint(unsigned ns) {
  g_tile_wait_hint.store(ns);
  return ok();
}

int atlas_debug_tile_unions(int on) {
  g_tile_unions.store(on ? 1 : 0);
  return ok();
}

int atlas_fvm_tile_union_groups(atlas_fvm_t h, int op, int dtype, int64_t* n) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (!n) return fail(ATLAS_EINVAL, "n is NULL");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (!valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "unsupported dtype %d", dtype);
  *n = 0;
  int rc = check_device(f);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(f->mu);
  rc = ensure_stencil(f, op, dtype);
  if (rc) return rc;
  rc = ensure_tile_layout(f, op, dtype);
  if (rc) return rc;
  const GroupTables& gt = f->st[op][dtype].grp;
  if (gt.ok) *n = gt.dev.union_groups;
  return ok();
}

int atlas_debug_tile_hang(int on) {
  g_tile_hang.store(on ? 1 : 0);
  return ok();
}

int atlas_fvm_group_table(atlas_fvm_t h, int op, int64_t* ngroups, int64_t* nent, int32_t* head, uint32_t* hdr,
                          double* w) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  atlasgb::Stencil s;
  atlasgb::GroupStencil gs;
  try {
    if (!atlasgb::build_stencil(f->mesh->m, f->d, op, s)) return fail(ATLAS_EINVAL, "stencil table overflow");
    if (!atlasgb::build_group_stencil(s, f->mesh->grid->g, gs))
      return fail(ATLAS_EINVAL, "this stencil has no node-group table");
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building operator tables");
  }
  const int64_t ng = static_cast<int64_t>(gs.first.size()) - 1, ne = static_cast<int64_t>(gs.hdr.size());
  if (ngroups) *ngroups = ng;
  if (nent) *nent = ne;
  if (head && ng) std::memcpy(head, gs.head.data(), sizeof(int32_t) * 4 * ng);
  if (hdr && ne) std::memcpy(hdr, gs.hdr.data(), sizeof(uint32_t) * ne);
  if (w && ne) {
    for (int64_t k = 0; k < ne * atlasgb::kGroup; ++k) {
      w[2 * k] = gs.w[gs.nw * k];
      w[2 * k + 1] = gs.nw == 2 ? gs.w[2 * k + 1] : 0.0;
    }
  }
  return ok();
}

int atlas_fvm_tile_table(atlas_fvm_t h, int op, int groups_per_tile, int rows_per_tile, int unions, int64_t* ntiles,
                         int64_t* nwords, int32_t* head, uint32_t* blob, int64_t* nunits, int64_t* unit_first,
                         int32_t* unit_tile) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (groups_per_tile < 1 || groups_per_tile > atlasgb::kTileMaxGroups)
    return fail(ATLAS_EINVAL, "groups_per_tile must be in [1, %d]", atlasgb::kTileMaxGroups);
  if (rows_per_tile < 1 || rows_per_tile > atlasgb::kMaxTileRows)
    return fail(ATLAS_EINVAL, "rows_per_tile must be in [1, %d]", atlasgb::kMaxTileRows);
  atlasgb::Stencil s;
  atlasgb::GroupStencil gs;
  atlasgb::TileStencil ts;
  try {
    if (!atlasgb::build_stencil(f->mesh->m, f->d, op, s)) return fail(ATLAS_EINVAL, "stencil table overflow");
    if (!atlasgb::build_group_stencil(s, f->mesh->grid->g, gs) ||
        !atlasgb::build_tile_stencil(gs, s, groups_per_tile, ts, unions != 0, rows_per_tile))
      return fail(ATLAS_EINVAL, "this stencil has no node-group tile table");
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building operator tables");
  }
  const int64_t nt = ts.ntiles, nw = static_cast<int64_t>(ts.blob.size());
  const int64_t nun = static_cast<int64_t>(ts.first.size()) - 1;
  if (ntiles) *ntiles = nt;
  if (nwords) *nwords = nw;
  if (nunits) *nunits = nun;
  if (head && nt) std::memcpy(head, ts.head.data(), sizeof(int32_t) * atlasgb::kTileHead * nt);
  if (blob && nw) std::memcpy(blob, ts.blob.data(), sizeof(uint32_t) * nw);
  if (unit_first) std::memcpy(unit_first, ts.first.data(), sizeof(int64_t) * (nun + 1));
  if (unit_tile) std::memcpy(unit_tile, ts.unit_tile.data(), sizeof(int32_t) * (nun + 1));
  return ok();
}

int atlas_fvm_stencil_table(atlas_fvm_t h, int op, int64_t* nnz, int* nin, int* nout, int32_t* ptr, int32_t* nbr,
                            double* w, double* b) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  atlasgb::Stencil s;
  try {
    if (!atlasgb::build_stencil(f->mesh->m, f->d, op, s)) return fail(ATLAS_EINVAL, "stencil table overflow");
  } catch (const std::bad_alloc&) {
    return fail(ATLAS_ENOMEM, "host allocation failed while building operator tables");
  }
  const size_t V = s.ptr.size() - 1, n = s.nbr.size();
  if (nnz) *nnz = static_cast<int64_t>(n);
  if (nin) *nin = s.nin;
  if (nout) *nout = s.nout;
  if (ptr) std::memcpy(ptr, s.ptr.data(), sizeof(int32_t) * (V + 1));
  if (nbr && n) std::memcpy(nbr, s.nbr.data(), sizeof(int32_t) * n);
  if (w && n) std::memcpy(w, s.w.data(), sizeof(double) * 2 * n);
  if (b) {
    if (s.has_b) std::memcpy(b, s.b.data(), sizeof(double) * 2 * V);
    else std::memset(b, 0, sizeof(double) * 2 * V);
  }
  return ok();
}

size_t atlas_fvm_integral_workspace_bytes(atlas_fvm_t h, int nlev) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f || nlev < 0) return 0;
  return static_cast<size_t>(std::max(f->num_sms, 1)) * 8 * static_cast<size_t>(nlev) * sizeof(double);
}

int atlas_fvm_integral(atlas_fvm_t h, const void* x, int64_t node0, int64_t count, int nlev, int64_t ld,
                       atlas_dtype dtype, double* out, void* ws, size_t ws_bytes, void* stream) {
  CallRange range_("atlas_fvm_integral");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (!valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "unknown dtype %d", static_cast<int>(dtype));
  const int64_t V = f->mesh->grid->g.nnodes;
  if (node0 < 0 || count < 0 || node0 + count > V)
    return fail(ATLAS_EINVAL, "node range [%lld, %lld) outside [0, %lld)", static_cast<long long>(node0),
                static_cast<long long>(node0 + count), static_cast<long long>(V));
  const void* used[1] = {x};
  int rc = check_field_args(dtype, nlev, ld, used, 1);
  if (rc) return rc;
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  if (reinterpret_cast<uintptr_t>(out) % 8 || reinterpret_cast<uintptr_t>(ws) % 8)
    return fail(ATLAS_EALIGN, "out and ws must be 8-byte aligned");
  const size_t need = atlas_fvm_integral_workspace_bytes(h, nlev);
  if (!ws && need > 0) return fail(ATLAS_EINVAL, "workspace pointer is NULL");
  if (ws_bytes < need) return fail(ATLAS_EINVAL, "workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
  rc = check_device(f);
  if (rc) return rc;
  if (nlev == 0) return ok();
  {
    std::lock_guard<std::mutex> lk(f->mu);
    if (!f->d_V) {
      cudaError_t err = cudaSuccess;
      f->d_V = f->vmem.upload(f->d.V, err);
      if (err != cudaSuccess) {
        f->vmem.release();
        f->d_V = nullptr;
        return err == cudaErrorMemoryAllocation ? fail(ATLAS_ENOMEM, "device allocation failed for the volumes")
                                                : cuda_fail(err, "upload of the volumes");
      }
    }
  }
  atlasgb::IntegralLaunch l;
  l.V = f->d_V + node0;
  l.x = x;
  l.count = static_cast<int32_t>(count);
  l.nlev = nlev;
  l.ld = ld;
  l.part = static_cast<double*>(ws);
  l.out = out;
  const int64_t maxb = static_cast<int64_t>(std::max(f->num_sms, 1)) * 8;
  if (count == 0) {
    l.nblocks = 1;  // the sums are 0: one block with no nodes writes them
    l.chunk = 0;
    l.count = 0;
  } else {
    const int64_t chunk = (count + maxb - 1) / maxb;
    l.chunk = static_cast<int32_t>(chunk);
    l.nblocks = static_cast<int32_t>((count + chunk - 1) / chunk);
  }
  cudaError_t e = atlasgb::launch_integral(storage_of(dtype), l, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "integral kernel launch");
  return ok();
}

void atlas_fvm_destroy(atlas_fvm_t h) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return;
  if (f->users > 0) {
    fail(ATLAS_ESTATE, "fvm still used by %d batch(es) or partition(s); not destroyed", f->users);
    return;
  }
  unreg(f);
  for (auto& row : f->st)
    for (auto& t : row) t.mem.release();
  for (auto& row : f->eg)
    for (auto& t : row) t.mem.release();
  f->vmem.release();
  f->mesh->users--;
  delete f;
}

int atlas_nabla_gradient(atlas_fvm_t fvm, const void* f, void* gx, void* gy, int nlev, int64_t ld, atlas_dtype dtype,
                         void* stream) {
  CallRange range_("atlas_nabla_gradient");
  return run_stencil_op(fvm, atlasgb::OP_GRAD, f, nullptr, gx, gy, nlev, ld, dtype, stream);
}
int atlas_nabla_divergence(atlas_fvm_t fvm, const void* u, const void* v, void* div, int nlev, int64_t ld,
                           atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_divergence");
  return run_stencil_op(fvm, atlasgb::OP_DIV, u, v, div, nullptr, nlev, ld, dtype, stream);
}
int atlas_nabla_laplacian(atlas_fvm_t fvm, const void* f, void* lap, int nlev, int64_t ld, atlas_dtype dtype,
                          void* stream) {
  CallRange range_("atlas_nabla_laplacian");
  return run_stencil_op(fvm, atlasgb::OP_LAP, f, nullptr, lap, nullptr, nlev, ld, dtype, stream);
}
int atlas_nabla_gradient_adjoint(atlas_fvm_t fvm, const void* gx, const void* gy, void* f, int nlev, int64_t ld,
                                 atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_gradient_adjoint");
  return run_stencil_op(fvm, atlasgb::OP_GRAD_ADJ, gx, gy, f, nullptr, nlev, ld, dtype, stream);
}
int atlas_nabla_divergence_adjoint(atlas_fvm_t fvm, const void* div, void* u, void* v, int nlev, int64_t ld,
                                   atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_divergence_adjoint");
  return run_stencil_op(fvm, atlasgb::OP_DIV_ADJ, div, nullptr, u, v, nlev, ld, dtype, stream);
}
int atlas_nabla_curl(atlas_fvm_t fvm, const void* u, const void* v, void* zeta, int nlev, int64_t ld,
                     atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_curl");
  return run_stencil_op(fvm, atlasgb::OP_CURL, u, v, zeta, nullptr, nlev, ld, dtype, stream);
}

int atlas_nabla_curl_adjoint(atlas_fvm_t fvm, const void* zeta, void* u, void* v, int nlev, int64_t ld,
                             atlas_dtype dtype, void* stream) {
  return run_stencil_op(fvm, atlasgb::OP_CURL_ADJ, zeta, nullptr, u, v, nlev, ld, dtype, stream);
}
int atlas_nabla_vector_gradient(atlas_fvm_t h, const void* u, const void* v, void* ux, void* uy, void* vx, void* vy,
                                int nlev, int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_vector_gradient");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  // the two launches must not see each other's outputs as inputs
  const void* ins[2] = {u, v};
  void* outs[4] = {ux, uy, vx, vy};
  for (int k = 0; k < 4; ++k)
    if (!outs[k]) return fail(ATLAS_EINVAL, "NULL output field");
  if (!u || !v) return fail(ATLAS_EINVAL, "NULL input field");
  if (valid_dtype(dtype) && ld >= 1 && ld <= kMaxLd) {
    const int rc = check_no_overlap(ins, 2, outs, 4, f->mesh->grid->g.nnodes * ld * elem_size(dtype));
    if (rc) return rc;
  }
  const int rc = run_stencil_op(h, atlasgb::OP_VGRAD, u, nullptr, ux, uy, nlev, ld, dtype, stream);
  if (rc) return rc;
  return run_stencil_op(h, atlasgb::OP_VGRAD, v, nullptr, vx, vy, nlev, ld, dtype, stream);
}

size_t atlas_nabla_workspace_bytes(atlas_fvm_t h, int op, int nlev, int64_t ld, atlas_dtype dtype) {
  atlas_fvm_s* f = get_fvm(h);
  if (!f || nlev < 0 || ld < nlev || ld < 1 || ld > kMaxLd || !valid_dtype(dtype)) return 0;
  if (op != ATLAS_OP_GRADIENT && op != ATLAS_OP_DIVERGENCE && op != ATLAS_OP_LAPLACIAN) return 0;
  return ws_layout(f, op, ld, dtype).total;
}

int atlas_nabla_gradient_edges(atlas_fvm_t h, const void* fin, void* gx, void* gy, void* ws, size_t ws_bytes, int nlev,
                               int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_gradient_edges");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (f->mesh->grid->g.regional())
    return fail(ATLAS_EINVAL, "the edge-based two-pass variant covers global grids only");
  if (dtype == ATLAS_BF16) return fail(ATLAS_EDTYPE, "the edge-based forms take F32 or F64 fields");
  const void* used[3] = {fin, gx, gy};
  int rc = check_field_args(dtype, nlev, ld, used, 3);
  if (rc) return rc;
  const void* ins[1] = {fin};
  void* outs[2] = {gx, gy};
  rc = check_no_overlap(ins, 1, outs, 2, f->mesh->grid->g.nnodes * ld * elem_size(dtype));
  if (rc) return rc;
  WsLayout w;
  rc = check_ws(f, ATLAS_OP_GRADIENT, ws, ws_bytes, ld, dtype, w);
  if (rc) return rc;
  rc = check_device(f);
  if (rc) return rc;
  if (nlev == 0) return ok();
  rc = run_edges_op(f, 0, fin, nullptr, gx, gy, static_cast<char*>(ws), w, nlev, ld, dtype,
                    static_cast<cudaStream_t>(stream));
  return rc ? rc : ok();
}

int atlas_nabla_gradient_edges_averaged(atlas_fvm_t h, const void* fin, void* gx, void* gy, void* ws, size_t ws_bytes,
                                        int nlev, int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_gradient_edges_averaged");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (f->mesh->grid->g.regional())
    return fail(ATLAS_EINVAL, "the edge-based two-pass variant covers global grids only");
  if (dtype == ATLAS_BF16) return fail(ATLAS_EDTYPE, "the edge-based forms take F32 or F64 fields");
  const void* used[3] = {fin, gx, gy};
  int rc = check_field_args(dtype, nlev, ld, used, 3);
  if (rc) return rc;
  const void* ins[1] = {fin};
  void* outs[2] = {gx, gy};
  rc = check_no_overlap(ins, 1, outs, 2, f->mesh->grid->g.nnodes * ld * elem_size(dtype));
  if (rc) return rc;
  WsLayout w;
  rc = check_ws(f, ATLAS_OP_GRADIENT, ws, ws_bytes, ld, dtype, w);
  if (rc) return rc;
  rc = check_device(f);
  if (rc) return rc;
  if (nlev == 0) return ok();
  rc = run_edges_op(f, 2, fin, nullptr, gx, gy, static_cast<char*>(ws), w, nlev, ld, dtype,
                    static_cast<cudaStream_t>(stream));
  return rc ? rc : ok();
}

int atlas_nabla_divergence_edges(atlas_fvm_t h, const void* u, const void* v, void* div, void* ws, size_t ws_bytes,
                                 int nlev, int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_divergence_edges");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (f->mesh->grid->g.regional())
    return fail(ATLAS_EINVAL, "the edge-based two-pass variant covers global grids only");
  if (dtype == ATLAS_BF16) return fail(ATLAS_EDTYPE, "the edge-based forms take F32 or F64 fields");
  const void* used[3] = {u, v, div};
  int rc = check_field_args(dtype, nlev, ld, used, 3);
  if (rc) return rc;
  const void* ins[2] = {u, v};
  void* outs[1] = {div};
  rc = check_no_overlap(ins, 2, outs, 1, f->mesh->grid->g.nnodes * ld * elem_size(dtype));
  if (rc) return rc;
  WsLayout w;
  rc = check_ws(f, ATLAS_OP_DIVERGENCE, ws, ws_bytes, ld, dtype, w);
  if (rc) return rc;
  rc = check_device(f);
  if (rc) return rc;
  if (nlev == 0) return ok();
  rc = run_edges_op(f, 1, u, v, div, nullptr, static_cast<char*>(ws), w, nlev, ld, dtype,
                    static_cast<cudaStream_t>(stream));
  return rc ? rc : ok();
}

int atlas_nabla_laplacian_edges(atlas_fvm_t h, const void* fin, void* lap, void* ws, size_t ws_bytes, int nlev,
                                int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_laplacian_edges");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (f->mesh->grid->g.regional())
    return fail(ATLAS_EINVAL, "the edge-based two-pass variant covers global grids only");
  if (dtype == ATLAS_BF16) return fail(ATLAS_EDTYPE, "the edge-based forms take F32 or F64 fields");
  const void* used[2] = {fin, lap};
  int rc = check_field_args(dtype, nlev, ld, used, 2);
  if (rc) return rc;
  const void* ins[1] = {fin};
  void* outs[1] = {lap};
  rc = check_no_overlap(ins, 1, outs, 1, f->mesh->grid->g.nnodes * ld * elem_size(dtype));
  if (rc) return rc;
  WsLayout w;
  rc = check_ws(f, ATLAS_OP_LAPLACIAN, ws, ws_bytes, ld, dtype, w);
  if (rc) return rc;
  rc = check_device(f);
  if (rc) return rc;
  if (nlev == 0) return ok();
  char* base = static_cast<char*>(ws);
  void* g0 = base + w.g0;
  void* g1 = base + w.g1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = run_edges_op(f, 0, fin, nullptr, g0, g1, base, w, nlev, ld, dtype, s);
  if (rc) return rc;
  rc = run_edges_op(f, 1, g0, g1, lap, nullptr, base, w, nlev, ld, dtype, s);
  return rc ? rc : ok();
}

// Two-pass Laplacian on the library's static scratch (see noalloc.cu): same
// kernels as atlas_nabla_laplacian_edges, no allocation of any kind.
int atlas_nabla_laplacian_edges_noalloc(atlas_fvm_t h, const void* fin, void* lap, int nlev, int64_t ld,
                                        atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_nabla_laplacian_edges_noalloc");
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (f->mesh->grid->g.regional())
    return fail(ATLAS_EINVAL, "the edge-based two-pass variant covers global grids only");
  if (dtype == ATLAS_BF16) return fail(ATLAS_EDTYPE, "the edge-based forms take F32 or F64 fields");
  const void* used[2] = {fin, lap};
  int rc = check_field_args(dtype, nlev, ld, used, 2);
  if (rc) return rc;
  const void* ins[1] = {fin};
  void* outs[1] = {lap};
  rc = check_no_overlap(ins, 1, outs, 1, f->mesh->grid->g.nnodes * ld * elem_size(dtype));
  if (rc) return rc;
  const WsLayout w = ws_layout(f, ATLAS_OP_LAPLACIAN, ld, dtype);
  if (w.total > atlasgb::noalloc_scratch_bytes())
    return fail(ATLAS_EINVAL, "this grid and ld need %zu bytes of scratch; the static scratch holds %zu bytes",
                w.total, atlasgb::noalloc_scratch_bytes());
  rc = check_device(f);
  if (rc) return rc;
  const int prec = prec_of(dtype);
  {
    std::lock_guard<std::mutex> lk(f->mu);
    if (!f->eg[0][prec].ready || !f->eg[1][prec].ready)
      return fail(ATLAS_ESTATE, "edge tables of this dtype are not on the device: call atlas_fvm_prepare with the "
                                "gradient and divergence bits first (this entry point allocates nothing)");
  }
  void* scratch = nullptr;
  cudaError_t e = atlasgb::noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
  if (nlev == 0) return ok();
  char* base = static_cast<char*>(scratch);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // one vector width for both passes: the second reads whole vectors of the
  // intermediate gradient exactly where the first wrote them
  const void* all[4] = {fin, lap, base + w.g0, base + w.g1};
  const int vec = pick_vec(dtype, ld, all, 4, 0);
  rc = run_edges_op(f, 0, fin, nullptr, base + w.g0, base + w.g1, base, w, nlev, ld, dtype, s, vec);
  if (rc) return rc;
  rc = run_edges_op(f, 1, base + w.g0, base + w.g1, lap, nullptr, base, w, nlev, ld, dtype, s, vec);
  return rc ? rc : ok();
}

int atlas_field_sync(void* dst, const void* src, size_t bytes, int direction, void* stream) {
  CallRange range_("atlas_field_sync");
  if (bytes == 0) return ok();
  if (!dst || !src) return fail(ATLAS_EINVAL, "NULL pointer");
  cudaMemcpyKind kind;
  switch (direction) {
    case 0: kind = cudaMemcpyHostToDevice; break;
    case 1: kind = cudaMemcpyDeviceToHost; break;
    case 2: kind = cudaMemcpyDeviceToDevice; break;
    default: return fail(ATLAS_EINVAL, "direction must be 0 (H2D), 1 (D2H) or 2 (D2D)");
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  return ok();
}

}  // extern "C"

// ============================================================= partitions
// A band partition: part p of nparts owns the consecutive rows [r0, r1) (a
// contiguous range of node ids, rows are numbered north to south) and reads
// a halo of `halo` rows on each side.  Neighbours of a node lie in its own
// row (ring and pole edges) or the adjacent rows, and the two-ring Laplacian
// reaches two rows away, so a halo of 1 (2 for the Laplacian) rows holds
// every value the own nodes need; those rows belong to the two adjacent
// parts (each part has at least `halo` rows), so one exchange with each of
// them refreshes the halo.
struct atlas_part_s {
  atlas_fvm_s* fvm = nullptr;
  int nparts = 1, part = 0, halo = 1;
  int r0 = 0, r1 = 0;
  int64_t own0 = 0, own1 = 0, halo0 = 0, halo1 = 0;
  int peer[2] = {-1, -1};
  int64_t send0[2] = {0, 0}, send1[2] = {0, 0}, recv0[2] = {0, 0}, recv1[2] = {0, 0};
};

extern "C" {

int atlas_part_create(atlas_fvm_t h, int nparts, int part, int halo_rings, atlas_part_t* out) {
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  atlas_fvm_s* f = get_fvm(h);
  if (!f) return fail(ATLAS_ESTATE, "invalid or destroyed fvm handle");
  if (halo_rings != 1 && halo_rings != 2) return fail(ATLAS_EINVAL, "halo_rings must be 1 or 2");
  const atlasgb::Grid& g = f->mesh->grid->g;
  const int nrows = g.nlat;
  if (nparts < 1 || part < 0 || part >= nparts) return fail(ATLAS_EINVAL, "need 0 <= part < nparts");
  if (static_cast<int64_t>(nparts) * halo_rings > nrows)
    return fail(ATLAS_EINVAL, "%d parts of at least %d rows do not fit %d rows", nparts, halo_rings, nrows);
  // boundaries: the row start nearest to an equal share of the nodes, kept
  // at least halo_rings rows apart and from both ends
  std::vector<int> b(static_cast<size_t>(nparts) + 1, 0);
  b[nparts] = nrows;
  for (int k = 1; k < nparts; ++k) {
    const double target = static_cast<double>(g.nnodes) * k / nparts;
    int r = static_cast<int>(std::lower_bound(g.off.begin(), g.off.end(), static_cast<int64_t>(target)) - g.off.begin());
    if (r > 0 && r <= nrows && target - g.off[r - 1] < g.off[r] - target) --r;
    r = std::max(r, b[k - 1] + halo_rings);
    r = std::min(r, nrows - (nparts - k) * halo_rings);
    b[k] = r;
  }
  atlas_part_s* p = new (std::nothrow) atlas_part_s();
  if (!p) return fail(ATLAS_ENOMEM, "out of host memory");
  p->fvm = f;
  p->nparts = nparts;
  p->part = part;
  p->halo = halo_rings;
  p->r0 = b[part];
  p->r1 = b[part + 1];
  p->own0 = g.off[p->r0];
  p->own1 = g.off[p->r1];
  p->halo0 = g.off[std::max(0, p->r0 - halo_rings)];
  p->halo1 = g.off[std::min(nrows, p->r1 + halo_rings)];
  if (part > 0) {  // rows above: the end of part - 1
    p->peer[0] = part - 1;
    p->send0[0] = p->own0;
    p->send1[0] = g.off[p->r0 + halo_rings];
    p->recv0[0] = p->halo0;
    p->recv1[0] = p->own0;
  }
  if (part + 1 < nparts) {  // rows below: the start of part + 1
    p->peer[1] = part + 1;
    p->send0[1] = g.off[p->r1 - halo_rings];
    p->send1[1] = p->own1;
    p->recv0[1] = p->own1;
    p->recv1[1] = p->halo1;
  }
  f->users++;
  reg(p);
  *out = reinterpret_cast<atlas_part_t>(p);
  return ok();
}

int atlas_part_info(atlas_part_t h, int64_t* own0, int64_t* own1, int64_t* halo0, int64_t* halo1) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed partition handle");
  const atlas_part_s* p = reinterpret_cast<const atlas_part_s*>(h);
  if (own0) *own0 = p->own0;
  if (own1) *own1 = p->own1;
  if (halo0) *halo0 = p->halo0;
  if (halo1) *halo1 = p->halo1;
  return ok();
}

int atlas_part_neighbour(atlas_part_t h, int side, int* peer, int64_t* send0, int64_t* send1, int64_t* recv0,
                         int64_t* recv1) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed partition handle");
  if (side != 0 && side != 1) return fail(ATLAS_EINVAL, "side must be 0 (the part before) or 1 (after)");
  const atlas_part_s* p = reinterpret_cast<const atlas_part_s*>(h);
  if (peer) *peer = p->peer[side];
  if (send0) *send0 = p->send0[side];
  if (send1) *send1 = p->send1[side];
  if (recv0) *recv0 = p->recv0[side];
  if (recv1) *recv1 = p->recv1[side];
  return ok();
}

int atlas_part_apply(atlas_part_t h, int op, const void* in0, const void* in1, void* out0, void* out1, int nlev,
                     int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_part_apply");
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed partition handle");
  atlas_part_s* p = reinterpret_cast<atlas_part_s*>(h);
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (op == atlasgb::OP_LAP && p->halo < 2) return fail(ATLAS_EINVAL, "the Laplacian needs a halo of 2 rows");
  if (!live(p->fvm)) return fail(ATLAS_ESTATE, "the partition's fvm was destroyed");
  return run_stencil_range(p->fvm, op, in0, in1, out0, out1, nlev, ld, dtype, stream, p->own0, p->own1 - p->own0,
                           p->halo0, p->halo1 - p->halo0);
}

int atlas_part_interior(atlas_part_t h, int64_t* inner0, int64_t* inner1) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed partition handle");
  const atlas_part_s* p = reinterpret_cast<const atlas_part_s*>(h);
  if (!live(p->fvm)) return fail(ATLAS_ESTATE, "the partition's fvm was destroyed");
  const atlasgb::Grid& g = p->fvm->mesh->grid->g;
  // a side with a neighbour gives up halo rows to the exchange
  const int r0 = p->peer[0] >= 0 ? p->r0 + p->halo : p->r0;
  const int r1 = p->peer[1] >= 0 ? p->r1 - p->halo : p->r1;
  const int64_t a = g.off[std::min(std::max(r0, p->r0), p->r1)];
  const int64_t b = g.off[std::min(std::max(r1, p->r0), p->r1)];
  if (inner0) *inner0 = a;
  if (inner1) *inner1 = std::max(a, b);  // empty when the part is thinner than its halos
  return ok();
}

int atlas_part_apply_nodes(atlas_part_t h, int op, const void* in0, const void* in1, void* out0, void* out1,
                           int64_t node0, int64_t count, int nlev, int64_t ld, atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_part_apply_nodes");
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed partition handle");
  atlas_part_s* p = reinterpret_cast<atlas_part_s*>(h);
  if (op < 0 || op >= atlasgb::OP_COUNT) return fail(ATLAS_EINVAL, "unknown operator %d", op);
  if (op == atlasgb::OP_LAP && p->halo < 2) return fail(ATLAS_EINVAL, "the Laplacian needs a halo of 2 rows");
  if (!live(p->fvm)) return fail(ATLAS_ESTATE, "the partition's fvm was destroyed");
  if (count < 0 || node0 < p->own0 || node0 + count > p->own1)
    return fail(ATLAS_EINVAL, "node range [%lld, %lld) outside the own range [%lld, %lld)",
                static_cast<long long>(node0), static_cast<long long>(node0 + count),
                static_cast<long long>(p->own0), static_cast<long long>(p->own1));
  if (!valid_dtype(dtype)) return fail(ATLAS_EDTYPE, "unknown dtype %d", static_cast<int>(dtype));
  // the output pointers address row node0 - own0 of the own-range fields
  const int64_t skip = (node0 - p->own0) * ld * elem_size(dtype);
  auto at = [&](void* q) -> void* { return q ? static_cast<void*>(static_cast<char*>(q) + skip) : nullptr; };
  return run_stencil_range(p->fvm, op, in0, in1, at(out0), at(out1), nlev, ld, dtype, stream, node0, count, p->halo0,
                           p->halo1 - p->halo0);
}

void atlas_part_destroy(atlas_part_t h) {
  if (!live(h)) return;
  atlas_part_s* p = reinterpret_cast<atlas_part_s*>(h);
  unreg(p);
  p->fvm->users--;
  delete p;
}

}  // extern "C"

// ============================================================== remapping
struct atlas_remap_s {
  atlas_mesh_s* src = nullptr;
  atlas_grid_s* dst = nullptr;
  int64_t ntgt = 0;
  std::vector<int32_t> nodes;   // [T][3]
  std::vector<double> weights;  // [T][3]
  int device = -1, num_sms = 0;
  std::mutex mu;
  bool ready[2] = {false, false};  // device tables: float weights, double weights
  const void* d_nodes[2] = {nullptr, nullptr};
  const void* d_w[2] = {nullptr, nullptr};
  DevAlloc mem[2];
};

extern "C" {

int atlas_remap_create(atlas_mesh_t sh, atlas_grid_t th, atlas_remap_t* out) {
  CallRange range_("atlas_remap_create");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!live(sh)) return fail(ATLAS_ESTATE, "invalid or destroyed mesh handle");
  if (!live(th)) return fail(ATLAS_ESTATE, "invalid or destroyed grid handle");
  atlas_mesh_s* m = reinterpret_cast<atlas_mesh_s*>(sh);
  atlas_grid_s* g = reinterpret_cast<atlas_grid_s*>(th);
  if (m->grid->g.regional())
    return fail(ATLAS_EINVAL, "the source of a remap must be a global mesh (a regional grid can be a target)");
  atlas_remap_s* r = new (std::nothrow) atlas_remap_s();
  if (!r) return fail(ATLAS_ENOMEM, "out of host memory");
  int64_t missed = 0;
  try {
    if (!atlasgb::build_remap(m->m, g->g.lonlat.data(), g->g.nnodes, r->nodes, r->weights, missed)) {
      delete r;
      return fail(ATLAS_EINVAL, "inconsistent source mesh");
    }
  } catch (const std::bad_alloc&) {
    delete r;
    return fail(ATLAS_ENOMEM, "out of host memory building the remap");
  }
  if (missed) {
    delete r;
    return fail(ATLAS_EINVAL, "%lld target points lie in the polar caps (no source triangle)",
                static_cast<long long>(missed));
  }
  if (g->g.nnodes >= (int64_t(1) << 31)) {
    delete r;
    return fail(ATLAS_EINVAL, "too many target points");
  }
  r->src = m;
  r->dst = g;
  r->ntgt = g->g.nnodes;
  int dev = -1;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    r->device = dev;
    cudaDeviceGetAttribute(&r->num_sms, cudaDevAttrMultiProcessorCount, dev);
  } else {
    cudaGetLastError();
  }
  m->users++;
  g->users++;
  reg(r);
  *out = reinterpret_cast<atlas_remap_t>(r);
  return ok();
}

int atlas_remap_info(atlas_remap_t h, int64_t* ntgt, const int32_t** nodes, const double** weights) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed remap handle");
  const atlas_remap_s* r = reinterpret_cast<const atlas_remap_s*>(h);
  if (ntgt) *ntgt = r->ntgt;
  if (nodes) *nodes = r->nodes.data();
  if (weights) *weights = r->weights.data();
  return ok();
}

int atlas_remap_apply(atlas_remap_t h, const void* src, void* dst, int nlev, int64_t ld_src, int64_t ld_dst,
                      atlas_dtype dtype, void* stream) {
  CallRange range_("atlas_remap_apply");
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed remap handle");
  atlas_remap_s* r = reinterpret_cast<atlas_remap_s*>(h);
  const void* used[2] = {src, dst};
  int rc = check_field_args(dtype, nlev, ld_src, used, 2);
  if (rc) return rc;
  if (ld_dst < nlev || ld_dst < 1 || ld_dst > kMaxLd)
    return fail(ATLAS_EINVAL, "ld_dst=%lld outside [max(nlev, 1), 2^31 - 1] (nlev=%d)",
                static_cast<long long>(ld_dst), nlev);
  const int64_t es = elem_size(dtype);
  const void* ins[1] = {src};
  void* outs[1] = {dst};
  rc = check_no_overlap2(ins, 1, r->src->grid->g.nnodes * ld_src * es, outs, 1, r->ntgt * ld_dst * es);
  if (rc) return rc;
  if (r->device < 0) return fail(ATLAS_ECUDA, "no CUDA device was available when this remap was built");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != r->device)
    return fail(ATLAS_ESTATE, "remap lives on device %d, current device is %d", r->device, cur);
  if (nlev == 0 || r->ntgt == 0) return ok();
  const int prec = dtype == ATLAS_F64 ? 1 : 0;
  {
    std::lock_guard<std::mutex> lk(r->mu);
    if (!r->ready[prec]) {
      cudaError_t err = cudaSuccess;
      std::vector<int32_t> n4(static_cast<size_t>(4 * r->ntgt), 0);
      for (int64_t t = 0; t < r->ntgt; ++t)
        for (int k = 0; k < 3; ++k) n4[4 * t + k] = r->nodes[3 * t + k];
      r->d_nodes[prec] = r->mem[prec].upload(n4, err);
      std::vector<double> w4(static_cast<size_t>(4 * r->ntgt), 0.0);
      for (int64_t t = 0; t < r->ntgt; ++t)
        for (int k = 0; k < 3; ++k) w4[4 * t + k] = r->weights[3 * t + k];
      if (err == cudaSuccess)
        r->d_w[prec] = prec ? static_cast<const void*>(r->mem[prec].upload(w4, err))
                            : static_cast<const void*>(r->mem[prec].upload(convert<float>(w4), err));
      if (err != cudaSuccess) {
        r->mem[prec].release();
        return err == cudaErrorMemoryAllocation ? fail(ATLAS_ENOMEM, "device allocation failed for remap tables")
                                                : cuda_fail(err, "upload of remap tables");
      }
      r->ready[prec] = true;
    }
  }
  atlasgb::RemapLaunch l;
  l.nodes = r->d_nodes[prec];
  l.weights = r->d_w[prec];
  l.src = src;
  l.dst = dst;
  l.ntgt = static_cast<int32_t>(r->ntgt);
  l.nlev = nlev;
  l.ld_src = ld_src;
  l.ld_dst = ld_dst;
  // one levels-per-thread width for both fields: the widest both allow
  l.vec = std::min(pick_vec(dtype, ld_src, used, 2, 0), pick_vec(dtype, ld_dst, used, 2, 0));
  const int64_t nvec = (nlev + l.vec - 1) / l.vec;
  if (r->ntgt * nvec >= (int64_t(1) << 31)) return fail(ATLAS_EINVAL, "targets * level-vectors must stay below 2^31");
  l.idx32 = r->src->grid->g.nnodes * ld_src < (int64_t(1) << 31) && r->ntgt * ld_dst < (int64_t(1) << 31);
  l.threads = 256;
  const int64_t need = (r->ntgt * nvec + l.threads - 1) / l.threads;
  l.blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(r->num_sms) * 8)));
  l.bd.hi = static_cast<int32_t>(r->src->grid->g.nnodes);
  l.bd.err = atlasgb::bounds_word();
  cudaError_t e = atlasgb::launch_remap(storage_of(dtype), l, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "remap kernel launch");
  const int brc = bounds_after(stream, "remap kernel");
  return brc ? brc : ok();
}

void atlas_remap_destroy(atlas_remap_t h) {
  if (!live(h)) return;
  atlas_remap_s* r = reinterpret_cast<atlas_remap_s*>(h);
  unreg(r);
  r->mem[0].release();
  r->mem[1].release();
  r->src->users--;
  r->dst->users--;
  delete r;
}

}  // extern "C"

// ================================================================= batches
struct atlas_batch_s {
  std::vector<atlas_fvm_s*> fvms;
  // fields large enough to fill the GPU many times over run as plain launches
  // with their operator's launch shape; the rest share the persistent launch
  struct Plain {
    atlas_fvm_s* f;
    int op;
    const void* in0;
    const void* in1;
    void* out0;
    void* out1;
    int nlev;
    int64_t ld;
  };
  std::vector<Plain> plain;
  atlas_dtype dtype = ATLAS_F32;
  atlasgb::BatchParams params;  // descriptor table, passed by value to every launch
  int ndesc = 0;
  int64_t ntiles = 0, node_levels = 0;
  int tile_items = 0, threads = 0, blocks = 0, device = -1, vec = 1;
  bool idx32 = true;
  StorageType st = atlasgb::ST_F32;
};

extern "C" {

int atlas_batch_create(const atlas_batch_desc* descs, int n, atlas_dtype dtype, const atlas_batch_tune* tune,
                       atlas_batch_t* out) {
  CallRange range_("atlas_batch_create");
  if (!out) return fail(ATLAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!descs || n < 1 || n > atlasgb::kBatchMaxDesc)
    return fail(ATLAS_EINVAL, "need 1..%d descriptors", atlasgb::kBatchMaxDesc);
  if (dtype != ATLAS_F32 && dtype != ATLAS_F64) return fail(ATLAS_EDTYPE, "batches take F32 or F64 fields");
  atlas_batch_tune t{0, 0, 0, 0, 0};
  if (tune) t = *tune;
  const int want_vec = t.vec > 0 ? t.vec : 16 / elem_size(dtype);
  if (want_vec != 1 && want_vec != 2 && want_vec != 4) return fail(ATLAS_EINVAL, "batch vec must be 1, 2 or 4");
  const int tile_items = t.tile_items > 0 ? t.tile_items : 1024;
  const int threads = t.threads > 0 ? t.threads : 256;
  if (t.plain_waves < -1) return fail(ATLAS_EINVAL, "plain_waves must be >= -1");
  // default: fields of four full waves and more run as plain launches (their
  // operators' own kernels, the node-group ones for FP32), the smaller ones
  // share the persistent launch, where they cost no launch and no tail of
  // their own; -1 puts every field in the persistent launch
  const int plain_waves = t.plain_waves == 0 ? 4 : t.plain_waves;
  if (threads < 64 || threads > 1024 || threads % 32) return fail(ATLAS_EINVAL, "bad thread count %d", threads);
  std::vector<atlasgb::BatchDescDev> hd;
  hd.reserve(static_cast<size_t>(n));
  std::vector<atlas_batch_s::Plain> plain;
  int64_t tiles = 0, nl = 0;
  // Tiles are drawn in table order: the costlier tiles (divergence, then more
  // levels) go first so that the cheap ones fill the end of the launch.  The
  // order changes no result: every item is computed once, by one thread.
  std::vector<int> order(static_cast<size_t>(n));
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const int oa = descs[a].op == ATLAS_OP_DIVERGENCE, oc = descs[c].op == ATLAS_OP_DIVERGENCE;
    if (oa != oc) return oa > oc;
    return descs[a].nlev > descs[c].nlev;
  });
  int device = -1;
  std::vector<atlas_fvm_s*> fv;
  // one levels-per-thread width for the whole batch: the widest every field allows
  int vec = want_vec;
  bool idx32 = true;
  for (int k = 0; k < n; ++k) {
    const atlas_batch_desc& d = descs[k];
    const bool grad = d.op == ATLAS_OP_GRADIENT;
    const void* used[3] = {d.in0, grad ? d.out0 : d.in1, grad ? d.out1 : d.out0};
    vec = std::min(vec, pick_vec(dtype, d.ld, used, 3, want_vec));
  }
  if (threads > atlasgb::kBatchMaxThreads)
    return fail(ATLAS_EINVAL, "batch threads must be <= %d", atlasgb::kBatchMaxThreads);
  for (int slot = 0; slot < n; ++slot) {
    const int k = order[slot];
    const atlas_batch_desc& d = descs[k];
    atlas_fvm_s* f = get_fvm(d.fvm);
    if (!f) return fail(ATLAS_ESTATE, "descriptor %d: invalid fvm handle", k);
    int rc = check_device(f);
    if (rc) return rc;
    if (device < 0) device = f->device;
    if (f->device != device) return fail(ATLAS_EINVAL, "descriptor %d: all fields must live on one device", k);
    const bool grad = d.op == ATLAS_OP_GRADIENT;
    if (!grad && d.op != ATLAS_OP_DIVERGENCE) return fail(ATLAS_EINVAL, "descriptor %d: op must be gradient or divergence", k);
    const void* used[3] = {d.in0, grad ? d.out0 : d.in1, grad ? d.out1 : d.out0};
    rc = check_field_args(dtype, d.nlev, d.ld, used, 3);
    if (rc) return fail(rc, "descriptor %d: %s", k, g_err.c_str());
    {
      std::lock_guard<std::mutex> lk(f->mu);
      rc = ensure_stencil(f, grad ? atlasgb::OP_GRAD : atlasgb::OP_DIV, dtype);
      if (rc) return rc;
    }
    const atlasgb::DevStencil& s = f->st[grad ? atlasgb::OP_GRAD : atlasgb::OP_DIV][dtype].dev;
    nl += static_cast<int64_t>(s.nnodes) * d.nlev;
    fv.push_back(f);
    // a field of at least plain_waves full waves of the GPU (2048 resident
    // threads per SM): its own launch costs little next to its work and runs
    // the plain kernel, which keeps its pointers in the parameter bank (the
    // persistent kernel holds them in registers, 48 against 40)
    const int64_t own_items = static_cast<int64_t>(s.nnodes) * ((d.nlev + vec - 1) / vec);
    if (plain_waves > 0 && own_items >= static_cast<int64_t>(f->num_sms) * 2048 * plain_waves) {
      plain.push_back(atlas_batch_s::Plain{f, grad ? atlasgb::OP_GRAD : atlasgb::OP_DIV, d.in0,
                                           grad ? nullptr : d.in1, d.out0, grad ? d.out1 : nullptr, d.nlev, d.ld});
      continue;
    }
    hd.emplace_back();
    atlasgb::BatchDescDev& o = hd.back();
    o.ptr = s.ptr;
    o.nbr = s.nbr;
    o.w = s.w;
    o.b = s.b;
    o.in0 = d.in0;
    o.in1 = grad ? nullptr : d.in1;
    o.out0 = d.out0;
    o.out1 = grad ? d.out1 : nullptr;
    o.ld = d.ld;
    o.nlev = d.nlev;
    o.nvec = (d.nlev + vec - 1) / vec;
    const int64_t items = static_cast<int64_t>(s.nnodes) * o.nvec;
    if (items >= (int64_t(1) << 31)) return fail(ATLAS_EINVAL, "descriptor %d too large", k);
    o.items = static_cast<int32_t>(items);
    o.op = grad ? 0 : 1;
    const atlasgb::Div32 dv = atlasgb::make_div32(static_cast<uint32_t>(o.nvec));
    o.div_m = dv.m;
    o.div_s1 = dv.s1;
    o.div_s2 = dv.s2;
    o.nnodes = s.nnodes;
    o.nnz = s.nnz;
    if (static_cast<int64_t>(s.nnodes) * d.ld >= (int64_t(1) << 31)) idx32 = false;
    o.tile0 = static_cast<int32_t>(tiles);
    tiles += (items + tile_items - 1) / tile_items;
    if (tiles >= (int64_t(1) << 30)) return fail(ATLAS_EINVAL, "too many tiles: raise tile_items");
  }
  atlas_batch_s* b = new (std::nothrow) atlas_batch_s();
  if (!b) return fail(ATLAS_ENOMEM, "out of host memory");
  std::memset(&b->params, 0, sizeof(b->params));
  b->params.ndesc = static_cast<int32_t>(hd.size());
  b->params.ntiles = static_cast<int32_t>(tiles);
  b->params.tile_items = tile_items;
  b->params.err = atlasgb::bounds_word();
  for (size_t k = 0; k < hd.size(); ++k) b->params.d[k] = hd[k];
  b->plain = plain;
  b->dtype = dtype;
  b->fvms = fv;
  for (atlas_fvm_s* f : fv) f->users++;
  b->ndesc = n;
  b->ntiles = tiles;
  b->node_levels = nl;
  b->tile_items = tile_items;
  b->threads = threads;
  b->st = storage_of(dtype);
  b->device = device;
  b->vec = vec;
  b->idx32 = idx32;
  int bps = atlasgb::batch_occupancy(b->st, vec, idx32, threads);
  if (t.blocks_per_sm > 0) bps = std::min(bps, t.blocks_per_sm);
  const int64_t blocks = std::min<int64_t>(static_cast<int64_t>(fv[0]->num_sms) * bps, std::max<int64_t>(tiles, 1));
  b->blocks = static_cast<int>(blocks);
  reg(b);
  *out = reinterpret_cast<atlas_batch_t>(b);
  return ok();
}

int atlas_batch_launch(atlas_batch_t h, void* stream) {
  CallRange range_("atlas_batch_launch");
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed batch handle");
  atlas_batch_s* b = reinterpret_cast<atlas_batch_s*>(h);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != b->device)
    return fail(ATLAS_ESTATE, "batch lives on device %d, current device is %d", b->device, cur);
  for (const atlas_batch_s::Plain& p : b->plain) {
    const int64_t V = p.f->mesh->grid->g.nnodes;
    const int rc = run_stencil_range(p.f, p.op, p.in0, p.in1, p.out0, p.out1, p.nlev, p.ld, b->dtype, stream, 0, V,
                                     0, V);
    if (rc) return rc;
  }
  if (b->ntiles == 0) return ok();
  cudaError_t e = atlasgb::launch_batch(b->st, b->vec, b->idx32, b->params, b->threads, b->blocks,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
  const int rc = bounds_after(stream, "batch kernel");
  return rc ? rc : ok();
}

int atlas_batch_info(atlas_batch_t h, int64_t* tiles, int64_t* node_levels) {
  if (!live(h)) return fail(ATLAS_ESTATE, "invalid or destroyed batch handle");
  atlas_batch_s* b = reinterpret_cast<atlas_batch_s*>(h);
  if (tiles) *tiles = b->ntiles;
  if (node_levels) *node_levels = b->node_levels;
  return ok();
}

void atlas_batch_destroy(atlas_batch_t h) {
  if (!live(h)) return;
  atlas_batch_s* b = reinterpret_cast<atlas_batch_s*>(h);
  unreg(b);
  for (atlas_fvm_s* f : b->fvms) f->users--;
  delete b;
}

}  // extern "C"
