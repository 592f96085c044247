// Shared-memory node-group stencil kernels (sm_103a) for FP32 and bfloat16
// fields: a TMA producer warp feeding consumer warps through shared memory.
//
// The node-stencil operators read, for every output value, the values of the
// node and of its 6-18 stencil neighbours at the same level.  With levels
// innermost one neighbour row is a contiguous run of nlev values, so the
// work is a sequence of row gathers.  Every input row leaves HBM about once
// (the rows of nearby latitudes stay in L2); what limits the per-node
// kernels is the L1 data pipe, one 128-byte line per cycle and SM, which
// their gathers use about twice per line of data: a warp spans two nodes and
// two rows that do not start on line boundaries, and each lane reads the CSR
// entry of its own node.  These kernels instead
//   * cut every grid row into tiles of up to eleven groups of four
//     consecutive nodes and let the host list, per tile, the node rows the
//     tile reads -- its own and all their neighbours -- as a few runs of
//     consecutive node ids (the rows above and below, the wrap of the row,
//     the antipodes of the polar rows);
//   * have one producer warp copy those runs, and the tile's table, from
//     global memory into shared memory with TMA bulk copies (cp.async.bulk,
//     completion counted in bytes on an mbarrier), up to four tiles ahead of
//     the consumers, so that the consumers read their rows from shared
//     memory, where a warp's 16-byte-per-lane load of a row costs exactly its
//     four lines, and each staged row serves every node of the tile that
//     needs it;
//   * give each consumer warp a group (or half a group: two of its nodes)
//     and all levels: lane l holds levels 4l .. 4l+3 of every row it reads
//     (part A) and level 128 + l (part B); the warp's nodes walk their own
//     stencil rows in step, which gives independent chains of arithmetic
//     per lane;
//   * take the row neighbours that belong to the same group from the
//     registers that hold the group's own values (their entries come first
//     in every row, at known offsets);
//   * with one warp per group, walk a group whose union of stencil rows
//     matches its operator's pattern (patterns.h; almost every group of an
//     octahedral grid) in union form: each distinct neighbour row is read
//     once and applied to every node of the group whose row holds it, the
//     pattern's masks compiled in.  A two-ring Laplacian group reads 30
//     rows instead of 62, a one-ring group 12 instead of 18 per field;
//     the other groups keep per-node rows;
//   * do the arithmetic on pairs of levels with the packed FP32 instructions
//     (__fadd2_rn, __ffma2_rn): each half rounds as the scalar instruction
//     does.
// Every node accumulates its terms in its stencil row's order with the same
// subtraction and fused multiply-add as the per-node kernels (the union
// order meets every node's terms in its row's order; a row shorter
// than its group's longest is padded with zero-weight terms of the node
// itself, which add exact zeros), so the results are bitwise those of the
// per-node kernels.  No atomics: deterministic.  Every wait on an mbarrier is
// bounded: past the limit the kernel records an error code in a device word
// that the host reads, waits (bounded again) for the copies it issued, and
// returns.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

#include <type_traits>

#include "bounds.cuh"
#include "geometry.h"
#include "kernels.h"
#include "patterns.h"

namespace atlasgb {
namespace grp {

// ---------------------------------------------------------------- values
// N levels of one node row as float: N/2 pairs (the operands of the
// packed f32x2 instructions) for even N, else one scalar.
template <int N, bool PAIRS = (N % 2 == 0)> struct Vals {
  float2 p[N / 2];
};
template <int N> struct Vals<N, false> {
  float s[N];
};
template <> struct Vals<0, true> {};

__device__ __forceinline__ float2 pk(float x, float y) { return make_float2(x, y); }

template <int N>
__device__ __forceinline__ void v_zero(Vals<N>& x) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) x.p[k] = make_float2(0.0f, 0.0f);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) x.s[k] = 0.0f;
  }
}
// d = x - y, as x + (-y) (the same IEEE operation) on pairs
template <int N>
__device__ __forceinline__ void v_sub(const Vals<N>& x, const Vals<N>& y, Vals<N>& d) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) d.p[k] = __fadd2_rn(x.p[k], make_float2(-y.p[k].x, -y.p[k].y));
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) d.s[k] = x.s[k] - y.s[k];
  }
}
// acc = fma(w, d, acc), w the same for every level, given as a pair {w, w}
// (a scalar part uses its first half)
template <int N>
__device__ __forceinline__ void v_fma(float2 ww, const Vals<N>& d, Vals<N>& acc) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) acc.p[k] = __ffma2_rn(ww, d.p[k], acc.p[k]);
  } else {
    const float w = ww.x;
#pragma unroll
    for (int k = 0; k < N; ++k) acc.s[k] = fmaf(w, d.s[k], acc.s[k]);
  }
}

// A lane's share of one node row: VA levels of part A and VB of part B.
template <int VA, int VB> struct Lv {
  Vals<VA> a;
  Vals<VB> b;
};
template <int VA, int VB>
__device__ __forceinline__ void lv_zero(Lv<VA, VB>& x) {
  v_zero<VA>(x.a);
  if constexpr (VB > 0) v_zero<VB>(x.b);
}
template <int VA, int VB>
__device__ __forceinline__ void lv_sub(const Lv<VA, VB>& x, const Lv<VA, VB>& y, Lv<VA, VB>& d) {
  v_sub<VA>(x.a, y.a, d.a);
  if constexpr (VB > 0) v_sub<VB>(x.b, y.b, d.b);
}
template <int VA, int VB>
__device__ __forceinline__ void lv_fma(float2 ww, const Lv<VA, VB>& d, Lv<VA, VB>& acc) {
  v_fma<VA>(ww, d.a, acc.a);
  if constexpr (VB > 0) v_fma<VB>(ww, d.b, acc.b);
}

// N consecutive values of storage type S, as float, from shared memory
// (32-bit shared-window address)
template <typename S, int N> struct Ld;
template <int N> struct Ld<float, N> {
  static __device__ __forceinline__ void run(uint32_t a, Vals<N>& v) {
    if constexpr (N == 4) {
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(v.p[0].x), "=f"(v.p[0].y), "=f"(v.p[1].x), "=f"(v.p[1].y)
                   : "r"(a));
    } else if constexpr (N == 2) {
      asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.p[0].x), "=f"(v.p[0].y) : "r"(a));
    } else {
      asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v.s[0]) : "r"(a));
    }
  }
};
template <int N> struct Ld<uint16_t, N> {
  // bfloat16 -> float is the 16-bit pattern shifted into the high half
  static __device__ __forceinline__ float2 two(uint32_t t) {
    return make_float2(__uint_as_float(t << 16), __uint_as_float(t & 0xffff0000u));
  }
  static __device__ __forceinline__ void run(uint32_t a, Vals<N>& v) {
    if constexpr (N == 4) {
      uint32_t x, y;
      asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(a));
      v.p[0] = two(x);
      v.p[1] = two(y);
    } else if constexpr (N == 2) {
      uint32_t x;
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(x) : "r"(a));
      v.p[0] = two(x);
    } else {
      unsigned short x;
      asm volatile("ld.shared.u16 %0, [%1];" : "=h"(x) : "r"(a));
      v.s[0] = __uint_as_float(static_cast<uint32_t>(x) << 16);
    }
  }
};

// N values stored whole: levels at or past nlev (the row's padding up to
// the end of the vector) are written as zeros.
template <int N>
__device__ __forceinline__ void v_unpack(const Vals<N>& v, float* e, int nvalid) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      e[2 * k] = 2 * k < nvalid ? v.p[k].x : 0.0f;
      e[2 * k + 1] = 2 * k + 1 < nvalid ? v.p[k].y : 0.0f;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) e[k] = k < nvalid ? v.s[k] : 0.0f;
  }
}
template <typename S, int N> struct St;
template <int N> struct St<float, N> {
  static __device__ __forceinline__ void run(float* __restrict__ p, const Vals<N>& v, int nvalid) {
    float e[N];
    v_unpack<N>(v, e, nvalid);
    if constexpr (N == 4) *reinterpret_cast<float4*>(p) = make_float4(e[0], e[1], e[2], e[3]);
    else if constexpr (N == 2) *reinterpret_cast<float2*>(p) = make_float2(e[0], e[1]);
    else *p = e[0];
  }
};
template <int N> struct St<uint16_t, N> {
  static __device__ __forceinline__ void run(uint16_t* __restrict__ p, const Vals<N>& v, int nvalid) {
    float f[N];
    v_unpack<N>(v, f, nvalid);
    uint16_t e[N];
#pragma unroll
    for (int k = 0; k < N; ++k) e[k] = __bfloat16_as_ushort(__float2bfloat16_rn(f[k]));
    if constexpr (N == 4) {
      uint2 r;
      memcpy(&r, e, 8);
      *reinterpret_cast<uint2*>(p) = r;
    } else if constexpr (N == 2) {
      uint32_t r;
      memcpy(&r, e, 4);
      *reinterpret_cast<uint32_t*>(p) = r;
    } else {
      *p = e[0];
    }
  }
};

// Lane layout of one level block starting at level lev0: part A levels
// lev0 + VA*lane .. + VA-1, part B levels lev0 + 32*VA + VB*lane .. + VB-1.
template <int VA, int VB> struct Layout {
  int offA, offB;  // first level of the lane's part A and part B
  __device__ __forceinline__ Layout(int lev0, int lane) : offA(lev0 + VA * lane), offB(lev0 + 32 * VA + VB * lane) {}
};

// One node row's share of this lane from the staged row in slot `slot`
// (rb bytes per staged row), given the lane's part A and part B addresses in
// slot 0 (baseA, baseB): one multiply-add per part and load.  Unconditional:
// lanes past nlev read the padding of the row, the next row or the stage's
// slack (in bounds of the block's shared memory) and those values are never
// stored.
template <typename S, int VA, int VB>
__device__ __forceinline__ void lv_load_at(uint32_t slot, uint32_t rb, uint32_t baseA, uint32_t baseB,
                                           Lv<VA, VB>& x) {
  Ld<S, VA>::run(slot * rb + baseA, x.a);
  if constexpr (VB > 0) Ld<S, VB>::run(slot * rb + baseB, x.b);
}
// Stores cover the levels below nstore: nlev rounded up to the widest
// vector the row layout allows, so the padding up to the end of the last
// 16-byte vector is zeroed whatever VA and VB the launch uses.
template <typename S, int VA, int VB>
__device__ __forceinline__ void lv_store(S* __restrict__ row, const Layout<VA, VB>& L, int nlev, int nstore,
                                         const Lv<VA, VB>& x) {
  if (L.offA < nstore) St<S, VA>::run(row + L.offA, x.a, nlev - L.offA);
  if constexpr (VB > 0)
    if (L.offB < nstore) St<S, VB>::run(row + L.offB, x.b, nlev - L.offB);
}

// N weight pairs {w, w} (8 N bytes, 16-byte aligned for N >= 2) from the
// staged table: warp-uniform shared loads (broadcasts).
template <int N> struct Wts { float2 w[N]; };
template <int N>
__device__ __forceinline__ void load_wts(uint32_t a, Wts<N>& r) {
  if constexpr (N == 1) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.w[0].x), "=f"(r.w[0].y) : "r"(a));
  } else {
#pragma unroll
    for (int k = 0; k < N; k += 2)
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                   : "=f"(r.w[k].x), "=f"(r.w[k].y), "=f"(r.w[k + 1].x), "=f"(r.w[k + 1].y)
                   : "r"(a + 8u * k));
  }
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds_u2(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ int4 lds_i4(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}

// ------------------------------------------------------------ union groups
// One term of one node: per input the difference x - x_node and the fused
// multiply-adds of its weights, in the per-node kernels' order (w0, w1: the
// node's weights towards the neighbour).
template <int NIN, int NOUT, int VA, int VB>
__device__ __forceinline__ void term(const Lv<VA, VB>& x0, const Lv<VA, VB>& x1, const Lv<VA, VB>& o0,
                                     const Lv<VA, VB>& o1, float w0, float w1, Lv<VA, VB>& a0, Lv<VA, VB>& a1) {
  Lv<VA, VB> d;
  lv_sub(x0, o0, d);
  lv_fma(pk(w0, w0), d, a0);
  if constexpr (NIN == 1 && NOUT == 2) {
    lv_fma(pk(w1, w1), d, a1);
  } else if constexpr (NIN == 2) {
    lv_sub(x1, o1, d);
    lv_fma(pk(w1, w1), d, a0);
  }
}

// Union entry E of pattern P (patterns.h): the rows x of its neighbour (or,
// for a node of the group, its values in xo) applied to every node whose
// mask bit is set, in node order.  wv holds the weight words WLO .. of the
// entry's chunk.
template <class P, int E, int WLO, int NW, int NIN, int NOUT, int VA, int VB, int NWV>
__device__ __forceinline__ void union_entry(const Lv<VA, VB> (&x)[NIN], const float (&wv)[NWV],
                                            const Lv<VA, VB> (&xo)[NIN][4], Lv<VA, VB> (&acc)[NOUT][4]) {
  if constexpr (E < P::U) {
    constexpr int msk = P::mask(E);
    constexpr int wb = pat::wbase<P>(E) * NW - WLO;
    int r = 0;
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
      if ((msk >> gg) & 1) {
        const int wi = wb + r * NW;
        if constexpr (pat::in_group<P>(E)) {
          constexpr int src = P::RUN0 + E;
          term<NIN, NOUT>(xo[0][src], xo[NIN - 1][src], xo[0][gg], xo[NIN - 1][gg], wv[wi], wv[wi + NW - 1],
                          acc[0][gg], acc[NOUT - 1][gg]);
        } else {
          term<NIN, NOUT>(x[0], x[NIN - 1], xo[0][gg], xo[NIN - 1][gg], wv[wi], wv[wi + NW - 1], acc[0][gg],
                          acc[NOUT - 1][gg]);
        }
        ++r;
      }
    }
  }
}
// the rows of union entry E from its staged slot (entries of the group's
// own nodes are not loaded)
template <class P, int E, typename S, int NIN, int VA, int VB>
__device__ __forceinline__ void union_load(uint32_t slot, uint32_t rb, const uint32_t (&baseA)[NIN],
                                           const uint32_t (&baseB)[NIN], Lv<VA, VB> (&x)[NIN]) {
  if constexpr (E < P::U && !pat::in_group<P>(E)) {
#pragma unroll
    for (int m = 0; m < NIN; ++m) lv_load_at<S, VA, VB>(slot, rb, baseA[m], baseB[m], x[m]);
  }
}
// Words of a union group's table: U slots, then the weights, each part
// padded to a multiple of four words.
template <class P, int NW>
__host__ __device__ constexpr int union_words() {
  return ((P::U + 3) & ~3) + ((pat::wbase<P>(P::U) * NW + 3) & ~3);
}

// The union walk of one group over one level block, four entries (chunk C)
// at a time: their slots (one 16-byte load), their weights, their rows,
// then the entries in order.  o_s: the group's slots; o_w: its weights.
template <class P, int C, typename S, int NIN, int NOUT, int NW, int VA, int VB>
__device__ __forceinline__ void union_walk(const uint32_t o_s, const uint32_t o_w, const uint32_t rb,
                                           const uint32_t (&baseA)[NIN], const uint32_t (&baseB)[NIN],
                                           const Lv<VA, VB> (&xo)[NIN][4], Lv<VA, VB> (&acc)[NOUT][4],
                                           const uint32_t slot_cap, const uint32_t own,
                                           unsigned long long* const bd_err, const int32_t t) {
  constexpr int E0 = 4 * C;
  constexpr int NE = P::U - E0 < 4 ? P::U - E0 : 4;
  constexpr int WLO = (pat::wbase<P>(E0) * NW) & ~3;
  constexpr int WHI = (pat::wbase<P>(E0 + NE) * NW + 3) & ~3;
  constexpr int NWV = WHI - WLO;
  const uint4 q = lds_u4(o_s + 16u * static_cast<uint32_t>(C));
  uint32_t sl[4] = {q.x, q.y, q.z, q.w};
  if constexpr (kBoundsCheck) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (!in_bounds(u >= NE || sl[u] < slot_cap, bd_err, BC_TILE_TABLE, t)) sl[u] = own;
  }
  float wv[NWV];
#pragma unroll
  for (int k = 0; k < NWV / 4; ++k) {
    const uint4 w4 = lds_u4(o_w + 4u * static_cast<uint32_t>(WLO + 4 * k));
    wv[4 * k] = __uint_as_float(w4.x);
    wv[4 * k + 1] = __uint_as_float(w4.y);
    wv[4 * k + 2] = __uint_as_float(w4.z);
    wv[4 * k + 3] = __uint_as_float(w4.w);
  }
  Lv<VA, VB> x[4][NIN];
  union_load<P, E0, S, NIN>(sl[0], rb, baseA, baseB, x[0]);
  union_load<P, E0 + 1, S, NIN>(sl[1], rb, baseA, baseB, x[1]);
  union_load<P, E0 + 2, S, NIN>(sl[2], rb, baseA, baseB, x[2]);
  union_load<P, E0 + 3, S, NIN>(sl[3], rb, baseA, baseB, x[3]);
  union_entry<P, E0, WLO, NW, NIN, NOUT>(x[0], wv, xo, acc);
  union_entry<P, E0 + 1, WLO, NW, NIN, NOUT>(x[1], wv, xo, acc);
  union_entry<P, E0 + 2, WLO, NW, NIN, NOUT>(x[2], wv, xo, acc);
  union_entry<P, E0 + 3, WLO, NW, NIN, NOUT>(x[3], wv, xo, acc);
  if constexpr (E0 + 4 < P::U)
    union_walk<P, C + 1, S, NIN, NOUT, NW, VA, VB>(o_s, o_w, rb, baseA, baseB, xo, acc, slot_cap, own, bd_err, t);
}

// ------------------------------------------------------------- mbarriers
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Wait until the phase with the given parity has completed, for at most
// `limit` SM clock cycles; false on time-out.  hint_ns > 0 lets each try
// suspend the thread for up to that many nanoseconds (fewer tries, a later
// wake-up); 0 tries with the hardware's own short suspension.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit, uint32_t hint_ns = 0) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    if (hint_ns)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(bar), "r"(parity), "r"(hint_ns)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// Bulk copy of bytes (a multiple of 16) from global src to shared dst (both
// 16-byte aligned), its completion counted on bar.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Error codes recorded in the device error word (bits); the word lives in
// group.cu and its device address travels in the kernel arguments.
constexpr unsigned kErrConsumerWait = 1u;  // a consumer gave up waiting for a tile
constexpr unsigned kErrProducerWait = 2u;  // the producer gave up waiting for a free buffer
constexpr unsigned kErrDrainWait = 4u;     // copies still in flight when the kernel gave up

struct TileArgs {
  const int32_t* head;    // [ntiles][kTileHead]
  const uint32_t* blob;   // per-tile tables
  const void* in0;
  const void* in1;
  void* out0;
  void* out1;
  int32_t t0, ntiles;     // tiles t0 .. t0 + ntiles - 1
  int32_t nlev, nstore, nlb;
  int64_t ld;
  uint32_t rows_bytes;    // bytes of one field's staged rows in a stage (slots cap * row bytes)
  uint32_t stage_bytes;   // bytes of one stage (NIN fields' rows, then the tile blob)
  int32_t nstages;        // 2 .. kMaxStages tiles in flight per block
  long long wait_limit;   // clock cycles any wait may take
  int32_t hang_test;      // 1: the consumers also wait on a barrier nothing completes (test of the time-out)
  uint32_t wait_hint_ns;  // suspension hint of the consumers' waits (0: none)
  unsigned* err;          // the device error word
  Bounds bd;              // bounds-checked build: input and output rows, blob words (nnz)
  int32_t max_groups;     // groups per tile of the table
};

constexpr int kMaxStages = 4;

// Block: NC consumer warps (warp 0 .. NC-1), then one producer warp.  Tiles
// t0 + blockIdx.x, + gridDim.x, ...; the block's k-th tile goes to stage
// k % nstages, the (k / nstages)-th use of that stage.
template <typename S, int NIN, int NOUT, bool HAS_B, int NW, int VA, int VB, int BATCH, int NPW>
__global__ void __launch_bounds__(NPW == 4 ? ((NIN == 1 && NOUT == 1) || (NIN == 1 && sizeof(S) == 2) ? 512 : 384)
                                            : 512,
                                  1)
    tile_kernel(const TileArgs a) {
  constexpr int LB = 32 * (VA + VB);  // levels per level block
  constexpr uint32_t ES = sizeof(S);
  // union pattern of the operator: the two-ring Laplacian or a one-ring table
  using UP = std::conditional_t<NIN == 1 && NOUT == 1, pat::Ring2, pat::Ring1>;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  const int ns = a.nstages;
  const uint32_t full0 = base + static_cast<uint32_t>(ns) * a.stage_bytes;  // full[4], empty[4], hang
  const uint32_t empty0 = full0 + 8 * kMaxStages;
  const uint32_t hang = empty0 + 8 * kMaxStages;
  const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31u);
  const int nc = static_cast<int>(blockDim.x >> 5) - 1;  // consumer warps
  if (threadIdx.x == 0) {
    for (int i = 0; i < ns; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, static_cast<uint32_t>(nc));
    }
    mbar_init(hang, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t row_bytes = a.ld * static_cast<int64_t>(ES);

  if (warp == nc) {
    // ------------------------------------------------------------ producer
    // The tile header: words 0..7 (two uniform 16-byte loads) and range
    // r = (first node, count, first slot, 0) in lane r.  The next tile's
    // header is requested before this tile's copies are issued, so its
    // latency hides behind the wait for a free stage.
    const int32_t t_end = a.t0 + a.ntiles;
    struct Head {
      int4 i0, i1, r;
    };
    auto load_head = [&](int32_t t) {
      const int4* h = reinterpret_cast<const int4*>(a.head + static_cast<int64_t>(t) * kTileHead);
      Head x;
      x.i0 = __ldg(h);
      x.i1 = __ldg(h + 1);
      x.r = lane < kTileRanges ? __ldg(h + 2 + lane) : make_int4(0, 0, 0, 0);
      return x;
    };
    int k = 0;
    bool ok = true;
    int32_t t = a.t0 + static_cast<int32_t>(blockIdx.x);
    Head cur{};
    if (t < t_end) cur = load_head(t);
    for (; t < t_end; t += static_cast<int32_t>(gridDim.x), ++k) {
      const int32_t tn = t + static_cast<int32_t>(gridDim.x);
      Head nxt{};
      if (tn < t_end) nxt = load_head(tn);
      const int st = k % ns;
      const uint32_t use = static_cast<uint32_t>(k / ns);
      const uint32_t full = full0 + 8 * st, empty = empty0 + 8 * st;
      const int32_t nranges = cur.i0.z, slots = cur.i0.w, boff = cur.i1.x, bbytes = cur.i1.y;
      if (k >= ns && ok) {
        // the consumers released this stage's previous tile
        bool got = true;
        if (lane == 0) got = mbar_wait(empty, (use - 1) & 1u, a.wait_limit);
        got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (!got) {
          if (lane == 0) atomicOr(a.err, kErrProducerWait);
          ok = false;
        }
      }
      if (!ok) break;
      const uint32_t sbase = base + static_cast<uint32_t>(st) * a.stage_bytes;
      if constexpr (kBoundsCheck) {
        // the header's sizes and copy ranges against the stage and the
        // field rows of the launch; a tile that fails is not copied: its
        // stage gets an empty table (no groups) and its barrier completes
        const bool hv = nranges >= 0 && nranges <= kTileRanges && slots >= 0 &&
                        static_cast<int64_t>(slots) * row_bytes <= a.rows_bytes && bbytes >= 16 && bbytes % 16 == 0 &&
                        static_cast<uint32_t>(NIN) * a.rows_bytes + static_cast<uint32_t>(bbytes) <= a.stage_bytes &&
                        boff >= 0 && 4ll * boff + bbytes / 4 <= a.bd.nnz;  // boff: 16-byte units
        const bool rv = lane >= nranges || (cur.r.y >= 0 && cur.r.x >= a.bd.lo &&
                                            static_cast<int64_t>(cur.r.x) + cur.r.y <= a.bd.hi && cur.r.z >= 0 &&
                                            cur.r.z + cur.r.y <= slots);
        if (!__all_sync(0xffffffffu, hv && rv)) {
          if (lane == 0) {
            in_bounds(false, a.bd.err, BC_TILE_HEAD, t);
            const uint32_t tb = sbase + static_cast<uint32_t>(NIN) * a.rows_bytes;
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(tb), "r"(0u) : "memory");
            mbar_expect_tx(full, 0u);
          }
          __syncwarp();
          cur = nxt;
          continue;
        }
      }
      if (lane == 0)
        mbar_expect_tx(full, static_cast<uint32_t>(NIN) * static_cast<uint32_t>(slots) * static_cast<uint32_t>(row_bytes) +
                                 static_cast<uint32_t>(bbytes));
      __syncwarp();
      if (lane < nranges) {
        const uint32_t bytes = static_cast<uint32_t>(cur.r.y) * static_cast<uint32_t>(row_bytes);
        const uint32_t dst = sbase + static_cast<uint32_t>(cur.r.z) * static_cast<uint32_t>(row_bytes);
        bulk_copy(dst, static_cast<const char*>(a.in0) + static_cast<int64_t>(cur.r.x) * row_bytes, bytes, full);
        if constexpr (NIN == 2)
          bulk_copy(dst + a.rows_bytes, static_cast<const char*>(a.in1) + static_cast<int64_t>(cur.r.x) * row_bytes,
                    bytes, full);
      }
      if (lane == 31)
        bulk_copy(sbase + static_cast<uint32_t>(NIN) * a.rows_bytes, a.blob + 4 * static_cast<int64_t>(boff),
                  static_cast<uint32_t>(bbytes), full);
      cur = nxt;
    }
    // before leaving, the copies of the last tiles must have landed (a
    // consumer may have given up early; the shared memory must not go away
    // under them)
    if (lane == 0) {
      for (int kk = (k >= ns ? k - ns : 0); kk < k; ++kk)
        if (!mbar_wait(full0 + 8 * (kk % ns), static_cast<uint32_t>(kk / ns) & 1u, a.wait_limit))
          atomicOr(a.err, kErrDrainWait);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  if (a.hang_test && !mbar_wait(hang, 0u, a.wait_limit)) {
    if (lane == 0) atomicOr(a.err, kErrConsumerWait);
    return;
  }
  int k = 0;
  for (int32_t t = a.t0 + static_cast<int32_t>(blockIdx.x); t < a.t0 + a.ntiles; t += static_cast<int32_t>(gridDim.x), ++k) {
    const int st = k % ns;
    if (!mbar_wait(full0 + 8 * st, static_cast<uint32_t>(k / ns) & 1u, a.wait_limit, a.wait_hint_ns)) {
      if (lane == 0) atomicOr(a.err, kErrConsumerWait);
      return;
    }
    const uint32_t sbase = base + static_cast<uint32_t>(st) * a.stage_bytes;
    const uint32_t blob = sbase + static_cast<uint32_t>(NIN) * a.rows_bytes;
    const int4 ti = lds_i4(blob);
    int ngt = ti.x;
    // bounds-checked build: the stage's table capacity and row slots
    const uint32_t blob_cap = a.stage_bytes - static_cast<uint32_t>(NIN) * a.rows_bytes;
    const uint32_t slot_cap = a.rows_bytes / static_cast<uint32_t>(row_bytes);
    if (!in_bounds(ngt >= 0 && ngt <= a.max_groups && 16u + 48u * static_cast<uint32_t>(ngt) <= blob_cap, a.bd.err,
                   BC_TILE_TABLE, t))
      ngt = 0;
    const uint32_t o_b = blob + 16u + 16u * static_cast<uint32_t>(ngt);
    uint32_t rows[2] = {sbase, sbase + a.rows_bytes};
    const uint32_t rb = static_cast<uint32_t>(row_bytes);
    // work items: (group, part); a part is NPW consecutive nodes of the
    // group (NPW = 4: one warp per group; NPW = 2: two warps per group)
    constexpr int PARTS = 4 / NPW;
    for (int item = warp; item < ngt * PARTS; item += nc) {
      const int g = item / PARTS, n0 = (item % PARTS) * NPW;
      const int4 gh = lds_i4(blob + 16u + 16u * static_cast<uint32_t>(g));
      const uint32_t slot0 = static_cast<uint32_t>(gh.x);
      const int count = gh.w & 0xffff;
      const bool regular = ((gh.w >> 16) & 1) != 0;  // the same for the whole warp
      const bool uni = ((gh.w >> 17) & 1) != 0;      // a union group (one warp per group only)
      const int32_t node0 = gh.z;                    // the group's first node
      const int D = (gh.w >> 20) & 0xff;             // entries: union length, or the longest row
      if (NPW != 4 && uni) {
        in_bounds(false, a.bd.err, BC_TILE_TABLE, t);
        continue;
      }
      if (!in_bounds(count <= 4 && (!regular || count == 4) && (!uni || (count == 4 && D == UP::U)) && gh.x >= 0 &&
                         slot0 + static_cast<uint32_t>(count) <= slot_cap && gh.y >= 0 &&
                         4ll * gh.y + (uni ? 4ll * union_words<UP, NW>() : (16ll + 32ll * NW) * D) <=
                             static_cast<long long>(blob_cap) &&
                         node0 >= a.bd.olo && static_cast<int64_t>(node0) + count <= a.bd.ohi,
                     a.bd.err, BC_TILE_TABLE, t))
        continue;
      const int cnt = count - n0;  // nodes of this part (warp-uniform)
      if (cnt <= 0) continue;
      for (int lb = 0; lb < a.nlb; ++lb) {
        const Layout<VA, VB> L(lb * LB, lane);
        // this lane's part A and part B addresses in slot 0 of each field
        uint32_t baseA[NIN], baseB[NIN];
#pragma unroll
        for (int m = 0; m < NIN; ++m) {
          baseA[m] = rows[m] + static_cast<uint32_t>(sizeof(S)) * static_cast<uint32_t>(L.offA);
          baseB[m] = rows[m] + static_cast<uint32_t>(sizeof(S)) * static_cast<uint32_t>(L.offB);
        }
        Lv<VA, VB> xo[NIN][NPW], acc[NOUT][NPW];
#pragma unroll
        for (int gg = 0; gg < NPW; ++gg) {
#pragma unroll
          for (int m = 0; m < NIN; ++m) {
            if (gg < cnt)  // warp-uniform
              lv_load_at<S, VA, VB>(slot0 + n0 + gg, rb, baseA[m], baseB[m], xo[m][gg]);
            else lv_zero(xo[m][gg]);
          }
#pragma unroll
          for (int c = 0; c < NOUT; ++c) lv_zero(acc[c][gg]);
        }
        // every node of the part walks its own stencil row, all in step
        // (independent sums); D entries each, BATCH at a time.  Entry e of
        // the group: slots [4] (16 bytes), weight pairs [4][NW]; this part
        // reads its NPW of them.
        const uint32_t o_s = blob + 4u * static_cast<uint32_t>(gh.y);
        const uint32_t o_ws = o_s + 16u * static_cast<uint32_t>(D);
        auto slots = [&](int e, uint32_t (&sls)[NPW]) {
          const uint32_t at = o_s + 16u * static_cast<uint32_t>(e) + 4u * static_cast<uint32_t>(n0);
          if constexpr (NPW == 4) {
            const uint4 sl = lds_u4(at);
            sls[0] = sl.x;
            sls[1] = sl.y;
            sls[2] = sl.z;
            sls[3] = sl.w;
          } else {
            const uint2 sl = lds_u2(at);
            sls[0] = sl.x;
            sls[1] = sl.y;
          }
          if constexpr (kBoundsCheck) {
#pragma unroll
            for (int gg = 0; gg < NPW; ++gg)
              if (!in_bounds(sls[gg] < slot_cap, a.bd.err, BC_TILE_TABLE, t)) sls[gg] = slot0;
          }
        };
        auto weights = [&](int e, Wts<NPW * NW>& W) {
          load_wts<NPW * NW>(o_ws + 32u * NW * static_cast<uint32_t>(e) + 8u * NW * static_cast<uint32_t>(n0), W);
        };
        auto step = [&](int e, Lv<VA, VB> (&x)[NPW][NIN], Wts<NPW * NW>& W) {
          uint32_t sls[NPW];
          slots(e, sls);
          weights(e, W);
#pragma unroll
          for (int gg = 0; gg < NPW; ++gg)
#pragma unroll
            for (int m = 0; m < NIN; ++m) lv_load_at<S, VA, VB>(sls[gg], rb, baseA[m], baseB[m], x[gg][m]);
        };
        auto use = [&](const Lv<VA, VB> (&x)[NPW][NIN], const Wts<NPW * NW>& W) {
#pragma unroll
          for (int gg = 0; gg < NPW; ++gg) {
            Lv<VA, VB> d;
            lv_sub(x[gg][0], xo[0][gg], d);
            if constexpr (NIN == 1 && NOUT == 1) {
              lv_fma(W.w[gg], d, acc[0][gg]);
            } else if constexpr (NIN == 1) {
              lv_fma(W.w[2 * gg], d, acc[0][gg]);
              lv_fma(W.w[2 * gg + 1], d, acc[1][gg]);
            } else {
              lv_fma(W.w[2 * gg], d, acc[0][gg]);
              lv_sub(x[gg][1], xo[1][gg], d);
              lv_fma(W.w[2 * gg + 1], d, acc[0][gg]);
            }
          }
        };
        bool walked = false;
        if constexpr (NPW == 4) {
          if (uni) {
            union_walk<UP, 0, S, NIN, NOUT, NW, VA, VB>(o_s, o_s + 4u * ((UP::U + 3) & ~3), rb, baseA, baseB, xo, acc,
                                                        slot_cap, slot0, a.bd.err, t);
            walked = true;
          }
        }
        int e = walked ? D : 0;
        if (regular && !walked) {
          // the first R entries of every node are its row neighbours at
          // offsets kOff: those inside this part are already in registers
          // (its own values xo), the others are read from shared memory
          constexpr int R = (NIN == 1 && NOUT == 1) ? 4 : 2;
          constexpr int kOff[4] = {R == 4 ? -2 : -1, R == 4 ? -1 : 1, 1, 2};
#pragma unroll
          for (int r = 0; r < R; ++r) {
            Lv<VA, VB> x[NPW][NIN];
            Wts<NPW * NW> W;
            uint32_t sls[NPW];
            slots(r, sls);
            weights(r, W);
#pragma unroll
            for (int gg = 0; gg < NPW; ++gg) {
              const int src = gg + kOff[r];
#pragma unroll
              for (int m = 0; m < NIN; ++m) {
                if (src >= 0 && src < NPW) x[gg][m] = xo[m][src];
                else lv_load_at<S, VA, VB>(sls[gg], rb, baseA[m], baseB[m], x[gg][m]);
              }
            }
            use(x, W);
          }
          e = R;
        }
        for (; e + BATCH <= D; e += BATCH) {
          Lv<VA, VB> x[BATCH][NPW][NIN];
          Wts<NPW * NW> W[BATCH];
#pragma unroll
          for (int u = 0; u < BATCH; ++u) step(e + u, x[u], W[u]);
#pragma unroll
          for (int u = 0; u < BATCH; ++u) use(x[u], W[u]);
        }
        for (; e < D; ++e) {
          Lv<VA, VB> x[NPW][NIN];
          Wts<NPW * NW> W;
          step(e, x, W);
          use(x, W);
        }
#pragma unroll
        for (int gg = 0; gg < NPW; ++gg) {
          if (gg < cnt) {
            if constexpr (HAS_B) {
              const float2 b =
                  lds_f2(o_b + 32u * static_cast<uint32_t>(g) + 8u * static_cast<uint32_t>(n0 + gg));
              if constexpr (NIN == 2) {
                lv_fma(pk(b.x, b.x), xo[0][gg], acc[0][gg]);
                lv_fma(pk(b.y, b.y), xo[1][gg], acc[0][gg]);
              } else {
                lv_fma(pk(b.x, b.x), xo[0][gg], acc[0][gg]);
                lv_fma(pk(b.y, b.y), xo[0][gg], acc[1][gg]);
              }
            }
            const int64_t o = static_cast<int64_t>(node0 + n0 + gg) * a.ld;
            lv_store<S, VA, VB>(static_cast<S*>(a.out0) + o, L, a.nlev, a.nstore, acc[0][gg]);
            if constexpr (NOUT == 2) lv_store<S, VA, VB>(static_cast<S*>(a.out1) + o, L, a.nlev, a.nstore, acc[1][gg]);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty0 + 8 * st);
  }
}

}  // namespace grp

// Kernel of (operator shape, level layout, table layout) for storage S; the
// instantiations live in group_f32.cu and group_bf16.cu.
namespace grp {
template <typename F>
inline cudaError_t with_shape(const DevTiles& d, F&& f) {
  if (d.nin == 1 && d.nout == 1) return f.template operator()<1, 1, false, 1>();
  if (d.nin == 1 && d.nout == 2 && !d.has_b) return f.template operator()<1, 2, false, 2>();
  if (d.nin == 1 && d.nout == 2) return f.template operator()<1, 2, true, 2>();
  if (d.nin == 2 && d.nout == 1 && d.has_b) return f.template operator()<2, 1, true, 2>();
  return cudaErrorInvalidValue;
}

template <typename S, int NIN, int NOUT, bool HAS_B, int NW, int NPW>
inline const void* kernel_of(int va, int vb) {
  // steps (entries of the warp's nodes) whose rows are requested together
  constexpr int BATCH = (NIN == 1 && NW == 1) ? 4 : 2;
#define ATLASGB_TILE(A, B)                                                                                    \
  if (va == A && vb == B)                                                                                     \
    return reinterpret_cast<const void*>(&tile_kernel<S, NIN, NOUT, HAS_B, NW, A, B, BATCH, NPW>);
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
  int va, vb, npw;
  const void* fn = nullptr;
  template <int NIN, int NOUT, bool HAS_B, int NW>
  cudaError_t operator()() {
    fn = npw == 2 ? kernel_of<S, NIN, NOUT, HAS_B, NW, 2>(va, vb) : kernel_of<S, NIN, NOUT, HAS_B, NW, 4>(va, vb);
    return fn ? cudaSuccess : cudaErrorInvalidValue;
  }
};
}  // namespace grp

// npw: nodes per consumer warp, 4 (one warp per group) or 2 (two warps per group)
const void* tile_fn_f32(const DevTiles& d, int va, int vb, int npw);
const void* tile_fn_bf16(const DevTiles& d, int va, int vb, int npw);

}  // namespace atlasgb
