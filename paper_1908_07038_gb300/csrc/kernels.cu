// CUDA kernels (sm_103a) of the nabla operators on field[node][level].
//
// The operators are sparse stencils: every output value needs the node's own
// value and those of its 6-7 edge neighbours (19 for the fused Laplacian), a
// few flops each.  The work is therefore bound by HBM traffic, not by
// arithmetic, and tensor cores have no role.  Design:
//   * one thread handles one (node, level-vector) item: VEC consecutive levels
//     of one node, loaded as one 16-byte (or narrower) vector; consecutive
//     threads take consecutive level vectors of the same node row, so a warp
//     reads whole 128-byte segments of a row (levels innermost);
//   * neighbour rows are re-read through the read-only path (ld.global.nc);
//     the rows of three adjacent latitudes are a few MB and stay in L2, so
//     each input value leaves HBM about once;
//   * the CSR row (neighbour id and weight pair) is the same for all level
//     vectors of a node and is served from L1 as a broadcast;
//   * fixed CSR summation order, no atomics: results are bitwise
//     deterministic and independent of the launch shape.
// The edge-flux / node-gather pair and the persistent batched kernel reuse
// the same per-item device functions.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

#include "bounds.cuh"
#include "kernels.h"

namespace atlasgb {
namespace {

// ---------------------------------------------------------------- storage
template <int BYTES> struct Raw;
template <> struct Raw<16> { using T = uint4; };
template <> struct Raw<8> { using T = uint2; };
template <> struct Raw<4> { using T = unsigned int; };
template <> struct Raw<2> { using T = unsigned short; };

// bfloat16 is carried as its 16-bit pattern (uint16_t) inside the kernels
template <typename S, typename A> struct Conv {
  static __device__ __forceinline__ A to(S x) { return static_cast<A>(x); }
  static __device__ __forceinline__ S from(A x) { return static_cast<S>(x); }
};
template <> struct Conv<uint16_t, float> {
  static __device__ __forceinline__ float to(uint16_t x) { return __uint_as_float(static_cast<uint32_t>(x) << 16); }
  static __device__ __forceinline__ uint16_t from(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
};

template <typename S, typename A, int VEC>
__device__ __forceinline__ void vload(const S* __restrict__ p, A (&out)[VEC]) {
  constexpr int BYTES = VEC * static_cast<int>(sizeof(S));
  using R = typename Raw<BYTES>::T;
  const R raw = __ldg(reinterpret_cast<const R*>(p));
  S e[VEC];
  memcpy(e, &raw, BYTES);
#pragma unroll
  for (int k = 0; k < VEC; ++k) out[k] = Conv<S, A>::to(e[k]);
}

template <typename S, typename A, int VEC>
__device__ __forceinline__ void vstore(S* __restrict__ p, const A (&v)[VEC], int nvalid) {
  constexpr int BYTES = VEC * static_cast<int>(sizeof(S));
  using R = typename Raw<BYTES>::T;
  // The last vector of a row may reach past nlev into the row's padding
  // (ld is a multiple of VEC whenever VEC > 1).  It is stored whole, with
  // zeros in the padding levels: a partly written sector would make L2 read
  // it from DRAM first.
  S e[VEC];
#pragma unroll
  for (int k = 0; k < VEC; ++k) e[k] = Conv<S, A>::from(k < nvalid ? v[k] : A(0));
  R raw;
  memcpy(&raw, e, BYTES);
  *reinterpret_cast<R*>(p) = raw;
}

// VEC values as loaded, converted to the accumulation type where they are
// used.  For bfloat16 storage this keeps a neighbour's level-vector in VEC/2
// registers instead of VEC: the batch of neighbour vectors a thread has in
// flight is what sets the register count, and with it the occupancy.
template <typename S, typename A, int VEC, bool PACKED = (sizeof(S) == 2 && VEC >= 2)> struct RawVec {
  A v[VEC];
  __device__ __forceinline__ void load(const S* __restrict__ p) { vload<S, A, VEC>(p, v); }
  __device__ __forceinline__ A operator[](int k) const { return v[k]; }
};
template <int VEC> struct RawVec<uint16_t, float, VEC, true> {
  uint32_t w[VEC / 2];
  __device__ __forceinline__ void load(const uint16_t* __restrict__ p) {
    using R = typename Raw<VEC * 2>::T;
    const R raw = __ldg(reinterpret_cast<const R*>(p));
    memcpy(w, &raw, VEC * 2);
  }
  // element 2m is the low half of word m (little-endian), 2m+1 the high half
  __device__ __forceinline__ float operator[](int k) const {
    return (k & 1) ? __uint_as_float(w[k >> 1] & 0xffff0000u) : __uint_as_float(w[k >> 1] << 16);
  }
};

template <typename A> struct Pair;
template <> struct Pair<float> {
  static __device__ __forceinline__ void load(const float* p, int64_t k, float& x, float& y) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p) + k);
    x = t.x;
    y = t.y;
  }
};
template <> struct Pair<double> {
  static __device__ __forceinline__ void load(const double* p, int64_t k, double& x, double& y) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p) + k);
    x = t.x;
    y = t.y;
  }
};

// One CSR entry of a node stencil: neighbour id and its weight(s).  Float
// tables of one-input operators are packed so that one aligned vector load
// returns the entry: {j, w} (8 bytes) for the scalar-weight Laplacian,
// {j, w0, w1, 0} (16 bytes) otherwise.  Two-input float tables and all double
// tables keep separate nbr[] and w[][2] arrays (measured faster there).
template <typename A, bool SCALAR_W, bool PACKED> struct Entry;
template <bool SCALAR_W> struct Entry<float, SCALAR_W, false> {
  static __device__ __forceinline__ void load(const int32_t* __restrict__ nbr, const float* __restrict__ w, int32_t q,
                                              int32_t& j, float& w0, float& w1) {
    j = __ldg(nbr + q);
    if constexpr (SCALAR_W) {
      w0 = __ldg(w + q);
      w1 = 0.0f;
    } else {
      Pair<float>::load(w, q, w0, w1);
    }
  }
};
template <bool SCALAR_W> struct Entry<float, SCALAR_W, true> {
  static __device__ __forceinline__ void load(const int32_t* __restrict__, const float* __restrict__ w, int32_t q,
                                              int32_t& j, float& w0, float& w1) {
    if constexpr (SCALAR_W) {
      const uint2 e = __ldg(reinterpret_cast<const uint2*>(w) + q);
      j = static_cast<int32_t>(e.x);
      w0 = __uint_as_float(e.y);
      w1 = 0.0f;
    } else {
      const uint4 e = __ldg(reinterpret_cast<const uint4*>(w) + q);
      j = static_cast<int32_t>(e.x);
      w0 = __uint_as_float(e.y);
      w1 = __uint_as_float(e.z);
    }
  }
};
template <bool SCALAR_W, bool PACKED> struct Entry<double, SCALAR_W, PACKED> {
  static __device__ __forceinline__ void load(const int32_t* __restrict__ nbr, const double* __restrict__ w, int32_t q,
                                              int32_t& j, double& w0, double& w1) {
    j = __ldg(nbr + q);
    if constexpr (SCALAR_W) {
      w0 = __ldg(w + q);
      w1 = 0.0;
    } else {
      Pair<double>::load(w, q, w0, w1);
    }
  }
};

// ------------------------------------------------------- node stencil item
// out_c(i) = sum_q sum_m W_cm(q) (x_m(nbr q) - x_m(i)) + sum_m B_cm(i) x_m(i)
//
// The CSR row is consumed BATCH entries at a time: first the BATCH neighbour
// ids and weights, then all BATCH neighbour level-vectors are requested
// before any is used.  A short last batch is padded with the node itself and
// a zero weight (d = 0, so the padding adds exactly 0), which keeps every
// load and FMA unconditional.  Accumulation follows the CSR order, so the
// result does not depend on BATCH or VEC.  IDX32 selects 32-bit element
// offsets (nnodes * ld < 2^31), which saves the 64-bit index arithmetic.
template <bool IDX32> struct IdxT { using T = int64_t; };
template <> struct IdxT<true> { using T = uint32_t; };

template <typename S, typename A, int NIN, int NOUT, int VEC, bool HAS_B, bool SCALAR_W, int BATCH, bool IDX32>
__device__ __forceinline__ void stencil_item(const int32_t* __restrict__ ptr, const int32_t* __restrict__ nbr,
                                             const A* __restrict__ w, const A* __restrict__ b,
                                             const S* __restrict__ in0, const S* __restrict__ in1,
                                             S* __restrict__ out0, S* __restrict__ out1, int64_t ld, int32_t nlev,
                                             int32_t i, int32_t lev0, const Bounds& bd) {
  using Idx = typename IdxT<IDX32>::T;
  const Idx ldx = static_cast<Idx>(ld);
  const Idx oi = static_cast<Idx>(i) * ldx + static_cast<Idx>(lev0);
  if (!in_bounds(i >= bd.lo && i < bd.hi && i >= bd.olo && i < bd.ohi, bd.err, BC_OUTPUT, i)) return;
  int32_t q0 = __ldg(ptr + i), q1 = __ldg(ptr + i + 1);
  if (!in_bounds(q0 >= 0 && q0 <= q1 && q1 <= bd.nnz, bd.err, BC_ROW, i)) q0 = q1 = 0;
  A xi0[VEC], xi1[VEC], acc0[VEC], acc1[VEC];
  vload<S, A, VEC>(in0 + oi, xi0);
  if constexpr (NIN == 2) vload<S, A, VEC>(in1 + oi, xi1);
#pragma unroll
  for (int k = 0; k < VEC; ++k) {
    acc0[k] = A(0);
    acc1[k] = A(0);
  }
  for (int32_t qb = q0; qb < q1; qb += BATCH) {
    int32_t jj[BATCH];
    A wa[BATCH], wb[BATCH];
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      const bool real = qb + t < q1;
      const int32_t q = real ? qb + t : qb;
      int32_t j;
      A x0, x1;
      Entry<A, SCALAR_W, (NIN == 1)>::load(nbr, w, q, j, x0, x1);
      if (real && !in_bounds(j >= bd.lo && j < bd.hi, bd.err, BC_NEIGHBOUR, q)) j = i;
      jj[t] = real ? j : i;
      wa[t] = real ? x0 : A(0);
      wb[t] = real ? x1 : A(0);
    }
    RawVec<S, A, VEC> xa[BATCH], xb[NIN == 2 ? BATCH : 1];
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      const Idx oj = static_cast<Idx>(jj[t]) * ldx + static_cast<Idx>(lev0);
      xa[t].load(in0 + oj);
      if constexpr (NIN == 2) xb[t].load(in1 + oj);
    }
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        if constexpr (NIN == 1) {
          const A d = xa[t][k] - xi0[k];
          acc0[k] = fma(wa[t], d, acc0[k]);
          if constexpr (NOUT == 2) acc1[k] = fma(wb[t], d, acc1[k]);
        } else {
          acc0[k] = fma(wa[t], xa[t][k] - xi0[k], acc0[k]);
          acc0[k] = fma(wb[t], xb[t][k] - xi1[k], acc0[k]);
        }
      }
    }
  }
  if constexpr (HAS_B) {
    A b0, b1;
    Pair<A>::load(b, i, b0, b1);
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      if constexpr (NIN == 2) {
        acc0[k] = fma(b0, xi0[k], acc0[k]);
        acc0[k] = fma(b1, xi1[k], acc0[k]);
      } else {
        acc0[k] = fma(b0, xi0[k], acc0[k]);
        acc1[k] = fma(b1, xi0[k], acc1[k]);
      }
    }
  }
  const int nvalid = nlev - lev0;
  vstore<S, A, VEC>(out0 + oi, acc0, nvalid);
  if constexpr (NOUT == 2) vstore<S, A, VEC>(out1 + oi, acc1, nvalid);
}

// The items of a launch are cut into tiles of `tile` consecutive items
// (a multiple of blockDim.x); block b takes tiles b, b + gridDim.x, ...  and
// its threads walk each tile in passes of blockDim.x items.  With tile =
// blockDim.x this is the plain grid-stride loop: all resident blocks work on
// one contiguous window of the fields, which keeps the DRAM pages and TLB
// entries in use few.  Longer tiles let a block walk consecutive nodes, so
// the neighbour rows that one pass loads are largely those the next pass
// needs and are still in the SM's L1.  Measured on O1280 x 137: tiles of 8
// to 64 passes help the bfloat16 operators; the FP32 and FP64 kernels run
// faster with their own grid-stride loop.
// The host keeps gridDim.x * tile below 2^31 + gridDim.x * blockDim.x, so no
// sum here overflows 32 bits.
template <typename F>
__device__ __forceinline__ void for_each_item(uint32_t total, uint32_t tile, F&& f) {
  // one counter: step by blockDim.x within a tile, jump to the block's next
  // tile after `passes` steps (items only grow, so the first item past
  // total ends the walk)
  const uint32_t passes = tile / blockDim.x;
  const uint32_t jump = (gridDim.x - 1) * tile;
  uint32_t p = 0;
  for (uint32_t item = blockIdx.x * tile + threadIdx.x; item < total; item += blockDim.x) {
    f(item);
    if (++p == passes) {
      p = 0;
      item += jump;
    }
  }
}

// n / d for a divisor fixed per launch: t = umulhi(m, n), q = (t + ((n - t) >> s1)) >> s2
// (branch-free unsigned division by an invariant integer; exact for all 32-bit n).
__device__ __forceinline__ uint32_t div_by(uint32_t n, Div32 d) {
  const uint32_t t = __umulhi(d.m, n);
  return (t + ((n - t) >> d.s1)) >> d.s2;
}

template <typename S, typename A, int NIN, int NOUT, int VEC, bool HAS_B, bool SCALAR_W, int BATCH, bool IDX32>
__global__ void __launch_bounds__(512) stencil_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ nbr,
                                                      const A* __restrict__ w, const A* __restrict__ b,
                                                      const S* __restrict__ in0, const S* __restrict__ in1,
                                                      S* __restrict__ out0, S* __restrict__ out1, int32_t node0,
                                                      int32_t count, int32_t nlev, int64_t ld, uint32_t nvec,
                                                      Div32 dv, uint32_t tile, Bounds bd) {
  // nodes node0 .. node0 + count - 1 (all nodes, or one partition's own)
  const uint32_t total = static_cast<uint32_t>(count) * nvec;  // host guarantees < 2^31
  auto body = [&](uint32_t item) {
    const uint32_t k = div_by(item, dv);
    const uint32_t v = item - k * nvec;
    stencil_item<S, A, NIN, NOUT, VEC, HAS_B, SCALAR_W, BATCH, IDX32>(
        ptr, nbr, w, b, in0, in1, out0, out1, ld, nlev, node0 + static_cast<int32_t>(k), static_cast<int32_t>(v * VEC),
        bd);
  };
  // FP32 and FP64 fields: a plain grid-stride loop, which measured 7-8%
  // faster than the tile walk for the one-ring operators (the tile length
  // does not apply); bfloat16 fields: the tile walk, 10-20% faster.
  if constexpr (sizeof(S) == 2) {
    for_each_item(total, tile, body);
  } else {
    (void)tile;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += stride) body(item);
  }
}

// ------------------------------------------------------------- edge pass
// OP 0 (gradient): flux0 = k1 (x_b - x_a), flux1 = k2 (x_b - x_a)
// OP 1 (divergence): flux0 = k1 (u_b - u_a) + k2 (v_b - v_a) + k3 v_a
// OP 2 (gradient, averaged form): flux0 = k1 (x_a + x_b), flux1 = k2 (x_a + x_b)
//   (the face value of the Green-Gauss sum; in FP32 its node sums cancel
//   terms of size |x| S / V to leave a gradient of size |x| / R)
//
// Both passes walk their items (edge or node, level-vector) one block-wide
// pass at a time.  The items of a pass belong to at most blockDim.x
// consecutive edges (nodes); their connectivity and coefficients are staged
// in shared memory by one cooperative, coalesced load between two barriers,
// and every thread then reads its own from there (the threads of one edge or
// node read the same words: broadcasts).  The loop bound depends only on the
// block, so all threads reach every barrier.  Launched with at most
// kEdgeThreads threads per block.
constexpr int kEdgeThreads = 256;
constexpr int kGatherStage = 2048;  // CSR entries staged per pass (else read from global memory)

template <typename S, typename A, int OP, int VEC>
__global__ void __launch_bounds__(kEdgeThreads) edge_flux_kernel(const int32_t* __restrict__ e2n,
                                                                 const A* __restrict__ coef,
                                                                 const S* __restrict__ in0, const S* __restrict__ in1,
                                                                 A* __restrict__ flux0, A* __restrict__ flux1,
                                                                 uint32_t nedges, int32_t nlev, int64_t ld,
                                                                 uint32_t nvec, Div32 dv, Bounds bd) {
  __shared__ int2 s_ab[kEdgeThreads];
  __shared__ A s_k[3][kEdgeThreads];
  const uint32_t total = nedges * nvec;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < total; base += stride) {
    const uint32_t last = min(base + blockDim.x, total) - 1;
    const uint32_t e0 = div_by(base, dv);
    const uint32_t ne = div_by(last, dv) - e0 + 1;  // <= blockDim.x
    __syncthreads();  // the previous pass has read its stage
    for (uint32_t t = threadIdx.x; t < ne; t += blockDim.x) {
      const int64_t e = static_cast<int64_t>(e0) + t;
      int2 ab = __ldg(reinterpret_cast<const int2*>(e2n) + e);
      if (!in_bounds(ab.x >= bd.lo && ab.x < bd.hi && ab.y >= bd.lo && ab.y < bd.hi, bd.err, BC_EDGE_END, e))
        ab = make_int2(bd.lo, bd.lo);
      s_ab[t] = ab;
      s_k[0][t] = __ldg(coef + 3 * e);
      s_k[1][t] = __ldg(coef + 3 * e + 1);
      if constexpr (OP == 1) s_k[2][t] = __ldg(coef + 3 * e + 2);
    }
    __syncthreads();
    const uint32_t item = base + threadIdx.x;
    if (item < total) {
      const uint32_t e = div_by(item, dv);
      const uint32_t le = e - e0;
      const int32_t lev0 = static_cast<int32_t>((item - e * nvec) * VEC);
      const int2 ab = s_ab[le];
      const A k1 = s_k[0][le], k2 = s_k[1][le];
      const int64_t oa = static_cast<int64_t>(ab.x) * ld + lev0, ob = static_cast<int64_t>(ab.y) * ld + lev0;
      const int64_t oe = static_cast<int64_t>(e) * ld + lev0;
      A xa[VEC], xb[VEC], f0[VEC];
      vload<S, A, VEC>(in0 + oa, xa);
      vload<S, A, VEC>(in0 + ob, xb);
      const int nvalid = nlev - lev0;
      if constexpr (OP == 0 || OP == 2) {
        A f1[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          const A d = OP == 0 ? xb[k] - xa[k] : xa[k] + xb[k];
          f0[k] = k1 * d;
          f1[k] = k2 * d;
        }
        vstore<A, A, VEC>(flux0 + oe, f0, nvalid);
        vstore<A, A, VEC>(flux1 + oe, f1, nvalid);
      } else {
        const A k3 = s_k[2][le];
        A ya[VEC], yb[VEC];
        vload<S, A, VEC>(in1 + oa, ya);
        vload<S, A, VEC>(in1 + ob, yb);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          A t = k1 * (xb[k] - xa[k]);
          t = fma(k2, yb[k] - ya[k], t);
          f0[k] = fma(k3, ya[k], t);
        }
        vstore<A, A, VEC>(flux0 + oe, f0, nvalid);
      }
    }
  }
}

// OP 0: out0 = (1/V) sum +-flux0, out1 = (cos/V) sum +-flux1
// OP 1: out0 = (1/V) sum flux0 + pole_coef * v_i
// The pass's nodes, CSR offsets, node coefficients and (when they fit in
// kGatherStage) CSR entries are staged in shared memory.
template <typename S, typename A, int OP, int VEC>
__global__ void __launch_bounds__(kEdgeThreads) node_gather_kernel(const int32_t* __restrict__ ptr,
                                                                   const int32_t* __restrict__ ent,
                                                                   const A* __restrict__ node,
                                                                   const A* __restrict__ flux0,
                                                                   const A* __restrict__ flux1,
                                                                   const S* __restrict__ vin, S* __restrict__ out0,
                                                                   S* __restrict__ out1, int32_t nnodes, int32_t nlev,
                                                                   int64_t ld, uint32_t nvec, Div32 dv, Bounds bd) {
  __shared__ int32_t s_ptr[kEdgeThreads + 1];
  __shared__ int32_t s_ent[kGatherStage];
  __shared__ A s_node[3][kEdgeThreads];
  const uint32_t total = static_cast<uint32_t>(nnodes) * nvec;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < total; base += stride) {
    const uint32_t last = min(base + blockDim.x, total) - 1;
    const uint32_t i0 = div_by(base, dv);
    const uint32_t nn = div_by(last, dv) - i0 + 1;  // <= blockDim.x
    __syncthreads();  // the previous pass has read its stage
    for (uint32_t t = threadIdx.x; t <= nn; t += blockDim.x) s_ptr[t] = __ldg(ptr + i0 + t);  // i0 + nn <= nnodes
    for (uint32_t t = threadIdx.x; t < nn; t += blockDim.x) {
      const int64_t i = static_cast<int64_t>(i0) + t;
      s_node[0][t] = __ldg(node + 3 * i);
      s_node[1][t] = __ldg(node + 3 * i + 1);
      s_node[2][t] = __ldg(node + 3 * i + 2);
    }
    __syncthreads();
    const int32_t qfirst = s_ptr[0];
    const int32_t nq = s_ptr[nn] - qfirst;
    // bounds-checked build: a pass whose entries leave the table is not staged
    const bool rows_ok = !kBoundsCheck || (qfirst >= 0 && nq >= 0 && static_cast<int64_t>(qfirst) + nq <= bd.nnz);
    const bool staged = rows_ok && nq <= kGatherStage;  // the same for the whole block
    if (staged)
      for (int32_t t = static_cast<int32_t>(threadIdx.x); t < nq; t += static_cast<int32_t>(blockDim.x))
        s_ent[t] = __ldg(ent + qfirst + t);
    __syncthreads();
    const uint32_t item = base + threadIdx.x;
    if (item < total) {
      const uint32_t i = div_by(item, dv);
      const uint32_t li = i - i0;
      const int32_t lev0 = static_cast<int32_t>((item - i * nvec) * VEC);
      A acc0[VEC], acc1[VEC];
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        acc0[k] = A(0);
        acc1[k] = A(0);
      }
      int32_t q0 = s_ptr[li], q1 = s_ptr[li + 1];
      if (!in_bounds(q0 >= 0 && q0 <= q1 && q1 <= bd.nnz && (!staged || (q0 >= qfirst && q1 - qfirst <= nq)), bd.err,
                     BC_ROW, i))
        q1 = q0;
      for (int32_t q = q0; q < q1; ++q) {
        const int32_t t = staged ? s_ent[q - qfirst] : __ldg(ent + q);
        if (!in_bounds((t >> 1) >= bd.lo && (t >> 1) < bd.hi, bd.err, BC_EDGE_ID, q)) continue;
        const int64_t oe = static_cast<int64_t>(t >> 1) * ld + lev0;
        A f[VEC];
        vload<A, A, VEC>(flux0 + oe, f);
        if (t & 1) {
#pragma unroll
          for (int k = 0; k < VEC; ++k) acc0[k] -= f[k];
        } else {
#pragma unroll
          for (int k = 0; k < VEC; ++k) acc0[k] += f[k];
        }
        if constexpr (OP == 0) {
          vload<A, A, VEC>(flux1 + oe, f);
          if (t & 1) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) acc1[k] -= f[k];
          } else {
#pragma unroll
            for (int k = 0; k < VEC; ++k) acc1[k] += f[k];
          }
        }
      }
      const A inv_v = s_node[0][li];
      const int64_t oi = static_cast<int64_t>(i) * ld + lev0;
      const int nvalid = nlev - lev0;
      if constexpr (OP == 0) {
        const A cos_v = s_node[1][li];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          acc0[k] *= inv_v;
          acc1[k] *= cos_v;
        }
        vstore<S, A, VEC>(out0 + oi, acc0, nvalid);
        vstore<S, A, VEC>(out1 + oi, acc1, nvalid);
      } else {
        const A pc = s_node[2][li];
        A vi[VEC];
        vload<S, A, VEC>(vin + oi, vi);
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc0[k] = fma(pc, vi[k], acc0[k] * inv_v);
        vstore<S, A, VEC>(out0 + oi, acc0, nvalid);
      }
    }
  }
}

// ------------------------------------------------------- persistent batch
// One launch covers a list of tiles: block b takes tiles b, b + gridDim.x,
// ...; tile t belongs to the descriptor d with tile0[d] <= t < tile0[d+1]
// (binary search) and covers tile_items consecutive (node, level-vector)
// items of that field.  All fields of a batch share one VEC; operators are
// gradient (1 in, 2 out) and divergence (2 in, 1 out, B term).
//
// The descriptor table is a __grid_constant__ kernel parameter, and the tile
// and descriptor indices depend only on blockIdx, so every per-field value
// (pointers, sizes, divisor) is the same across the block and is read from
// the parameter space, as a plain launch reads its own arguments.  Copied to
// shared memory and held in per-thread registers, the same values cost a
// quarter of the gradient's throughput (measured: the register count capped
// occupancy at half the SM).  The gradient requests 6 neighbour vectors at a
// time and the divergence 3 (its two inputs make 6 loads), which keeps the
// kernel within 48 registers at 5 blocks of 256 threads per SM.
template <typename S, typename A, int VEC, bool IDX32>
__global__ void __launch_bounds__(256, 5) batch_kernel(const __grid_constant__ BatchParams P) {
  for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
    int lo = 0, hi = P.ndesc - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.d[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const BatchDescDev& D = P.d[lo];
    const Div32 dv{D.div_m, D.div_s1, D.div_s2};
    Bounds bd;
    if constexpr (kBoundsCheck) {
      bd.hi = bd.ohi = D.nnodes;
      bd.nnz = D.nnz;
      bd.err = P.err;
    }
    const uint32_t it0 = static_cast<uint32_t>(t - D.tile0) * static_cast<uint32_t>(P.tile_items);
    const uint32_t it1 = min(it0 + static_cast<uint32_t>(P.tile_items), static_cast<uint32_t>(D.items));
    for (uint32_t u = it0 + threadIdx.x; u < it1; u += blockDim.x) {
      const uint32_t i = div_by(u, dv);
      const int32_t lev0 = static_cast<int32_t>((u - i * static_cast<uint32_t>(D.nvec)) * VEC);
      if (D.op == 0)
        stencil_item<S, A, 1, 2, VEC, false, false, 6, IDX32>(
            D.ptr, D.nbr, static_cast<const A*>(D.w), static_cast<const A*>(D.b), static_cast<const S*>(D.in0),
            static_cast<const S*>(D.in1), static_cast<S*>(D.out0), static_cast<S*>(D.out1), D.ld, D.nlev,
            static_cast<int32_t>(i), lev0, bd);
      else
        stencil_item<S, A, 2, 1, VEC, true, false, 3, IDX32>(
            D.ptr, D.nbr, static_cast<const A*>(D.w), static_cast<const A*>(D.b), static_cast<const S*>(D.in0),
            static_cast<const S*>(D.in1), static_cast<S*>(D.out0), static_cast<S*>(D.out1), D.ld, D.nlev,
            static_cast<int32_t>(i), lev0, bd);
    }
  }
}

// ------------------------------------------------- volume-weighted integral
// I_k = sum over nodes i of V_i x_{i,k}, in FP64, for every level k (the
// global conservation sums: I of the divergence vanishes on the sphere).
// Pass 1: block b sums nodes [b chunk, (b + 1) chunk) of the range; thread t
// owns levels t, t + blockDim.x, ... and reads its level of each node row
// (consecutive threads, consecutive levels), accumulating with four
// interleaved FP64 accumulators (accumulator m takes the nodes congruent to
// m mod 4 in order, the tail goes to the first; combined as
// (a0 + a1) + (a2 + a3)) into part[b][k].  Pass 2: out[k] = the
// sum of part[b][k] in block order.  No atomics: the result is the same on
// every run and for every stream.
// binary32 -> binary64 from the IEEE-754 layouts, on the integer pipe: sign
// kept; a normal exponent is rebiased by 1023 - 127; a subnormal is
// normalised (shifted left by its leading zeros, exponent 897 - shift);
// zeros stay zeros, infinities and NaNs take exponent 2047 with the
// significand (payload) kept.  Exact for every input, branch-free; the
// conversion instruction would occupy GB300's narrow FP64 pipe, which the
// FMA of the sum needs.
__device__ __forceinline__ double widen(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const uint32_t lz = static_cast<uint32_t>(__clz(static_cast<int>(m | 1u))) - 8u;
  const bool sub = e == 0u;
  const uint32_t E = sub ? (m != 0u ? 897u - lz : 0u) : (e == 0xffu ? 2047u : e + (1023u - 127u));
  const uint32_t M = sub ? ((m << lz) & 0x7fffffu) : m;
  const uint32_t hi = (u & 0x80000000u) | (E << 20) | (M >> 3);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(M << 29));
}

template <typename S>
__device__ __forceinline__ double as_f64(const S* __restrict__ x, int64_t q) {
  if constexpr (sizeof(S) == 8)
    return __ldg(reinterpret_cast<const double*>(x) + q);
  else
    return widen(Conv<S, float>::to(x[q]));
}

template <typename S>
__global__ void __launch_bounds__(256) integral_partial_kernel(const double* __restrict__ V, const S* __restrict__ x,
                                                               int32_t count, int32_t chunk, int32_t nlev, int64_t ld,
                                                               double* __restrict__ part) {
  const int32_t n0 = blockIdx.x * chunk;
  const int32_t n1 = min(n0 + chunk, count);
  for (int32_t k = threadIdx.x; k < nlev; k += blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int32_t i = n0;
    // eight rows in flight per thread; accumulator m takes nodes i + m and
    // i + 4 + m, in that order
    for (; i + 7 < n1; i += 8) {
      double xv[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) xv[m] = as_f64(x, static_cast<int64_t>(i + m) * ld + k);
      a0 = fma(__ldg(V + i), xv[0], a0);
      a1 = fma(__ldg(V + i + 1), xv[1], a1);
      a2 = fma(__ldg(V + i + 2), xv[2], a2);
      a3 = fma(__ldg(V + i + 3), xv[3], a3);
      a0 = fma(__ldg(V + i + 4), xv[4], a0);
      a1 = fma(__ldg(V + i + 5), xv[5], a1);
      a2 = fma(__ldg(V + i + 6), xv[6], a2);
      a3 = fma(__ldg(V + i + 7), xv[7], a3);
    }
    for (; i < n1; ++i) a0 = fma(__ldg(V + i), as_f64(x, static_cast<int64_t>(i) * ld + k), a0);
    part[static_cast<int64_t>(blockIdx.x) * nlev + k] = (a0 + a1) + (a2 + a3);
  }
}

__global__ void __launch_bounds__(256) integral_final_kernel(const double* __restrict__ part, int32_t nblocks,
                                                             int32_t nlev, double* __restrict__ out) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nlev; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t b = 0; b < nblocks; ++b) s += part[static_cast<int64_t>(b) * nlev + k];
    out[k] = s;
  }
}

// ------------------------------------------------------------- remapping
// Linear interpolation in 3D on the sphere from a source mesh to target
// points: dst[t][k] = w0 src[n0][k] + w1 src[n1][k] + w2 src[n2][k], one
// (target, level-vector) item per thread.  The target's three nodes and
// weights (tn[t] = {n0, n1, n2, 0}, tw[t] = {w0, w1, w2, 0}) are the same
// for the items of a warp; the three source rows are requested together.
template <typename S, typename A, int VEC, bool IDX32>
__global__ void __launch_bounds__(512) remap_kernel(const int4* __restrict__ tn, const A* __restrict__ tw,
                                                    const S* __restrict__ src, S* __restrict__ dst, int32_t ntgt,
                                                    int32_t nlev, int64_t ld_src, int64_t ld_dst, uint32_t nvec,
                                                    Div32 dv, Bounds bd) {
  using Idx = typename IdxT<IDX32>::T;
  const uint32_t total = static_cast<uint32_t>(ntgt) * nvec;  // host guarantees < 2^31
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += stride) {
    const uint32_t t = div_by(item, dv);
    const int32_t lev0 = static_cast<int32_t>((item - t * nvec) * VEC);
    int4 n = __ldg(tn + t);
    if (!in_bounds(n.x >= bd.lo && n.x < bd.hi && n.y >= bd.lo && n.y < bd.hi && n.z >= bd.lo && n.z < bd.hi, bd.err,
                   BC_REMAP, t))
      n = make_int4(bd.lo, bd.lo, bd.lo, 0);
    const A w0 = __ldg(tw + 4 * static_cast<Idx>(t)), w1 = __ldg(tw + 4 * static_cast<Idx>(t) + 1),
            w2 = __ldg(tw + 4 * static_cast<Idx>(t) + 2);
    A x0[VEC], x1[VEC], x2[VEC], y[VEC];
    vload<S, A, VEC>(src + static_cast<Idx>(n.x) * static_cast<Idx>(ld_src) + static_cast<Idx>(lev0), x0);
    vload<S, A, VEC>(src + static_cast<Idx>(n.y) * static_cast<Idx>(ld_src) + static_cast<Idx>(lev0), x1);
    vload<S, A, VEC>(src + static_cast<Idx>(n.z) * static_cast<Idx>(ld_src) + static_cast<Idx>(lev0), x2);
#pragma unroll
    for (int k = 0; k < VEC; ++k) y[k] = fma(w2, x2[k], fma(w1, x1[k], w0 * x0[k]));
    vstore<S, A, VEC>(dst + static_cast<Idx>(t) * static_cast<Idx>(ld_dst) + static_cast<Idx>(lev0), y, nlev - lev0);
  }
}

// ------------------------------------------------------- FP64 FMA rate
// Eight independent chains of FP64 fused multiply-adds per thread,
// x <- x b + a (b < 1: the values stay bounded), iters steps each: 16 iters
// flops per thread, enough independent work to keep the FP64 pipe of every
// SM busy.  The sum of the chains is stored so nothing is optimised away.
__global__ void __launch_bounds__(256) fp64_fma_kernel(double* __restrict__ out, int64_t iters) {
  const int t = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
  const double a = 1.0e-3 + 1.0e-12 * t, b = 0.999999;
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0e-3 * k + 1.0e-9 * t;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], b, a);
  }
  out[t] = ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
}

// ---------------------------------------------------------------- dispatch
template <typename S, typename A, int NIN, int NOUT, int VEC, bool HAS_B, bool SCALAR_W, int BATCH>
cudaError_t run_stencil(const DevStencil& s, const StencilLaunch& l, cudaStream_t stream) {
  const uint32_t nvec = static_cast<uint32_t>((l.nlev + VEC - 1) / VEC);
  const Div32 dv = make_div32(nvec);
  const bool idx32 = static_cast<int64_t>(s.nnodes) * l.ld < (int64_t(1) << 31);
  if (idx32)
    stencil_kernel<S, A, NIN, NOUT, VEC, HAS_B, SCALAR_W, BATCH, true><<<l.blocks, l.threads, 0, stream>>>(
        s.ptr, s.nbr, static_cast<const A*>(s.w), static_cast<const A*>(s.b), static_cast<const S*>(l.in0),
        static_cast<const S*>(l.in1), static_cast<S*>(l.out0), static_cast<S*>(l.out1), l.node0, l.count, l.nlev, l.ld,
        nvec, dv, l.tile, l.bd);
  else
    stencil_kernel<S, A, NIN, NOUT, VEC, HAS_B, SCALAR_W, BATCH, false><<<l.blocks, l.threads, 0, stream>>>(
        s.ptr, s.nbr, static_cast<const A*>(s.w), static_cast<const A*>(s.b), static_cast<const S*>(l.in0),
        static_cast<const S*>(l.in1), static_cast<S*>(l.out0), static_cast<S*>(l.out1), l.node0, l.count, l.nlev, l.ld,
        nvec, dv, l.tile, l.bd);
  return cudaGetLastError();
}

template <typename S, typename A, int NIN, int NOUT, int VEC, bool HAS_B, bool SCALAR_W, int BATCH>
const void* stencil_fn() {
  return reinterpret_cast<const void*>(&stencil_kernel<S, A, NIN, NOUT, VEC, HAS_B, SCALAR_W, BATCH, true>);
}

// Visit the kernel instantiation of (storage, shape, vec); F is called with a
// tag carrying the template arguments.
template <typename S, typename A, int VEC, int BATCH, typename F>
auto with_shape(const DevStencil& s, F&& f) {
  if (s.scalar_w) return f.template operator()<S, A, 1, 1, VEC, false, true, BATCH>();
  if (s.nin == 1 && s.nout == 2 && !s.has_b) return f.template operator()<S, A, 1, 2, VEC, false, false, BATCH>();
  if (s.nin == 1 && s.nout == 2) return f.template operator()<S, A, 1, 2, VEC, true, false, BATCH>();
  return f.template operator()<S, A, 2, 1, VEC, true, false, BATCH>();
}

template <typename S, typename A, int VEC, typename F>
auto with_batch(const DevStencil& s, int batch, F&& f) {
  if (batch == 3) return with_shape<S, A, VEC, 3>(s, f);
  return with_shape<S, A, VEC, 6>(s, f);
}

template <typename S, typename A, typename F>
auto with_vec(const DevStencil& s, int vec, int batch, F&& f) {
  constexpr int maxvec = 16 / static_cast<int>(sizeof(S));
  if (vec >= 8 && maxvec >= 8) return with_batch<S, A, (maxvec >= 8 ? 8 : 1)>(s, batch, f);
  if (vec >= 4 && maxvec >= 4) return with_batch<S, A, (maxvec >= 4 ? 4 : 1)>(s, batch, f);
  if (vec >= 2) return with_batch<S, A, 2>(s, batch, f);
  return with_batch<S, A, 1>(s, batch, f);
}

template <typename F>
auto with_storage(StorageType st, const DevStencil& s, int vec, int batch, F&& f) {
  if (st == ST_F64) return with_vec<double, double>(s, vec, batch, f);
  if (st == ST_BF16) return with_vec<uint16_t, float>(s, vec, batch, f);
  return with_vec<float, float>(s, vec, batch, f);
}

struct RunStencil {
  const DevStencil& s;
  const StencilLaunch& l;
  cudaStream_t stream;
  template <typename S, typename A, int NIN, int NOUT, int VEC, bool HAS_B, bool SCALAR_W, int BATCH>
  cudaError_t operator()() const {
    return run_stencil<S, A, NIN, NOUT, VEC, HAS_B, SCALAR_W, BATCH>(s, l, stream);
  }
};

struct StencilFn {
  template <typename S, typename A, int NIN, int NOUT, int VEC, bool HAS_B, bool SCALAR_W, int BATCH>
  const void* operator()() const {
    return stencil_fn<S, A, NIN, NOUT, VEC, HAS_B, SCALAR_W, BATCH>();
  }
};

}  // namespace

// The bounds checks' device word pair {code, index} (bounds.cuh).
__device__ unsigned long long g_bounds[2];

bool bounds_checked() { return kBoundsCheck; }

unsigned long long* bounds_word() {
  if (!kBoundsCheck) return nullptr;
  static void* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!addr[dev] && cudaGetSymbolAddress(&addr[dev], g_bounds) != cudaSuccess) addr[dev] = nullptr;
  return static_cast<unsigned long long*>(addr[dev]);
}

cudaError_t bounds_error(unsigned long long* code, long long* index, bool clear) {
  unsigned long long w[2] = {0, 0};
  cudaError_t e = cudaMemcpyFromSymbol(w, g_bounds, sizeof(w));
  if (e != cudaSuccess) return e;
  *code = w[0];
  *index = static_cast<long long>(w[1]);
  if (clear && w[0] != 0) {
    const unsigned long long z[2] = {0, 0};
    e = cudaMemcpyToSymbol(g_bounds, z, sizeof(z));
  }
  return e;
}

// Host: multiplier and shifts of the branch-free division by d (d >= 1).
Div32 make_div32(uint32_t d) {
  Div32 r{0, 0, 0};
  if (d <= 1) return r;
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;  // ceil(log2 d)
  const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
  r.m = static_cast<uint32_t>(m);
  r.s1 = 1;
  r.s2 = l - 1;
  return r;
}

cudaError_t launch_stencil(StorageType st, const DevStencil& s, const StencilLaunch& l, cudaStream_t stream) {
  return with_storage(st, s, l.vec, l.batch, RunStencil{s, l, stream});
}

int stencil_occupancy(StorageType st, const DevStencil& s, int vec, int batch, int threads) {
  const void* fn = with_storage(st, s, vec, batch, StencilFn{});
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, 0) != cudaSuccess) return 1;
  return blocks > 0 ? blocks : 1;
}

namespace {
template <typename S, typename A, int VEC>
cudaError_t run_edges(int op, const DevEdges& e, const void* in0, const void* in1, void* flux0, void* flux1,
                      int32_t nlev, int64_t ld, int threads, int blocks, cudaStream_t stream) {
  const uint32_t nvec = static_cast<uint32_t>((nlev + VEC - 1) / VEC);
  const Div32 dv = make_div32(nvec);
  const A* coef = static_cast<const A*>(e.coef);
  Bounds bd;
  bd.hi = bd.ohi = e.nnodes;
  bd.err = bounds_word();
  if (op == 0)
    edge_flux_kernel<S, A, 0, VEC><<<blocks, threads, 0, stream>>>(
        e.e2n, coef, static_cast<const S*>(in0), nullptr, static_cast<A*>(flux0), static_cast<A*>(flux1),
        static_cast<uint32_t>(e.nedges), nlev, ld, nvec, dv, bd);
  else if (op == 2)
    edge_flux_kernel<S, A, 2, VEC><<<blocks, threads, 0, stream>>>(
        e.e2n, coef, static_cast<const S*>(in0), nullptr, static_cast<A*>(flux0), static_cast<A*>(flux1),
        static_cast<uint32_t>(e.nedges), nlev, ld, nvec, dv, bd);
  else
    edge_flux_kernel<S, A, 1, VEC><<<blocks, threads, 0, stream>>>(
        e.e2n, coef, static_cast<const S*>(in0), static_cast<const S*>(in1), static_cast<A*>(flux0), nullptr,
        static_cast<uint32_t>(e.nedges), nlev, ld, nvec, dv, bd);
  return cudaGetLastError();
}
template <typename S, typename A, int VEC>
cudaError_t run_gather(int op, const DevEdges& e, const void* flux0, const void* flux1, const void* vin, void* out0,
                       void* out1, int32_t nlev, int64_t ld, int threads, int blocks, cudaStream_t stream) {
  const uint32_t nvec = static_cast<uint32_t>((nlev + VEC - 1) / VEC);
  const Div32 dv = make_div32(nvec);
  const A* node = static_cast<const A*>(e.node);
  Bounds bd;  // input rows: the edges' fluxes; entries: the node->edge table
  bd.hi = static_cast<int32_t>(e.nedges);
  bd.ohi = e.nnodes;
  bd.nnz = e.nent;
  bd.err = bounds_word();
  if (op == 0)
    node_gather_kernel<S, A, 0, VEC><<<blocks, threads, 0, stream>>>(
        e.ptr, e.ent, node, static_cast<const A*>(flux0), static_cast<const A*>(flux1), nullptr, static_cast<S*>(out0),
        static_cast<S*>(out1), e.nnodes, nlev, ld, nvec, dv, bd);
  else
    node_gather_kernel<S, A, 1, VEC><<<blocks, threads, 0, stream>>>(
        e.ptr, e.ent, node, static_cast<const A*>(flux0), nullptr, static_cast<const S*>(vin), static_cast<S*>(out0),
        nullptr, e.nnodes, nlev, ld, nvec, dv, bd);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_edge_flux(StorageType st, int op, const DevEdges& e, const void* in0, const void* in1, void* flux0,
                             void* flux1, int32_t nlev, int64_t ld, int vec, int threads, int blocks,
                             cudaStream_t stream) {
  if (st == ST_F64) {
    if (vec >= 2) return run_edges<double, double, 2>(op, e, in0, in1, flux0, flux1, nlev, ld, threads, blocks, stream);
    return run_edges<double, double, 1>(op, e, in0, in1, flux0, flux1, nlev, ld, threads, blocks, stream);
  }
  if (st == ST_F32) {
    if (vec >= 4) return run_edges<float, float, 4>(op, e, in0, in1, flux0, flux1, nlev, ld, threads, blocks, stream);
    if (vec >= 2) return run_edges<float, float, 2>(op, e, in0, in1, flux0, flux1, nlev, ld, threads, blocks, stream);
    return run_edges<float, float, 1>(op, e, in0, in1, flux0, flux1, nlev, ld, threads, blocks, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_node_gather(StorageType st, int op, const DevEdges& e, const void* flux0, const void* flux1,
                               const void* vin, void* out0, void* out1, int32_t nlev, int64_t ld, int vec, int threads,
                               int blocks, cudaStream_t stream) {
  if (st == ST_F64) {
    if (vec >= 2) return run_gather<double, double, 2>(op, e, flux0, flux1, vin, out0, out1, nlev, ld, threads, blocks, stream);
    return run_gather<double, double, 1>(op, e, flux0, flux1, vin, out0, out1, nlev, ld, threads, blocks, stream);
  }
  if (st == ST_F32) {
    if (vec >= 4) return run_gather<float, float, 4>(op, e, flux0, flux1, vin, out0, out1, nlev, ld, threads, blocks, stream);
    if (vec >= 2) return run_gather<float, float, 2>(op, e, flux0, flux1, vin, out0, out1, nlev, ld, threads, blocks, stream);
    return run_gather<float, float, 1>(op, e, flux0, flux1, vin, out0, out1, nlev, ld, threads, blocks, stream);
  }
  return cudaErrorInvalidValue;
}

namespace {
template <bool IDX32>
const void* batch_fn_t(StorageType st, int vec) {
  if (st == ST_F64)
    return vec >= 2 ? reinterpret_cast<const void*>(&batch_kernel<double, double, 2, IDX32>)
                    : reinterpret_cast<const void*>(&batch_kernel<double, double, 1, IDX32>);
  if (vec >= 4) return reinterpret_cast<const void*>(&batch_kernel<float, float, 4, IDX32>);
  if (vec >= 2) return reinterpret_cast<const void*>(&batch_kernel<float, float, 2, IDX32>);
  return reinterpret_cast<const void*>(&batch_kernel<float, float, 1, IDX32>);
}
const void* batch_fn(StorageType st, int vec, bool idx32) {
  return idx32 ? batch_fn_t<true>(st, vec) : batch_fn_t<false>(st, vec);
}
}  // namespace

namespace {
template <typename S, typename A, int VEC, bool IDX32>
cudaError_t run_remap(const RemapLaunch& r, cudaStream_t stream) {
  const uint32_t nvec = static_cast<uint32_t>((r.nlev + VEC - 1) / VEC);
  remap_kernel<S, A, VEC, IDX32><<<r.blocks, r.threads, 0, stream>>>(
      static_cast<const int4*>(r.nodes), static_cast<const A*>(r.weights), static_cast<const S*>(r.src),
      static_cast<S*>(r.dst), r.ntgt, r.nlev, r.ld_src, r.ld_dst, nvec, make_div32(nvec), r.bd);
  return cudaGetLastError();
}
template <typename S, typename A, int MAXVEC, bool IDX32>
cudaError_t remap_vec(const RemapLaunch& r, cudaStream_t stream) {
  if (r.vec >= 8 && MAXVEC >= 8) return run_remap<S, A, (MAXVEC >= 8 ? 8 : 1), IDX32>(r, stream);
  if (r.vec >= 4 && MAXVEC >= 4) return run_remap<S, A, (MAXVEC >= 4 ? 4 : 1), IDX32>(r, stream);
  if (r.vec >= 2 && MAXVEC >= 2) return run_remap<S, A, (MAXVEC >= 2 ? 2 : 1), IDX32>(r, stream);
  return run_remap<S, A, 1, IDX32>(r, stream);
}
template <bool IDX32>
cudaError_t remap_st(StorageType st, const RemapLaunch& r, cudaStream_t stream) {
  if (st == ST_F64) return remap_vec<double, double, 2, IDX32>(r, stream);
  if (st == ST_BF16) return remap_vec<uint16_t, float, 8, IDX32>(r, stream);
  return remap_vec<float, float, 4, IDX32>(r, stream);
}
}  // namespace

cudaError_t launch_integral(StorageType st, const IntegralLaunch& l, cudaStream_t stream) {
  if (l.count < 0 || l.nlev <= 0 || l.nblocks <= 0) return cudaSuccess;
  const int threads = l.nlev >= 256 ? 256 : ((l.nlev + 31) / 32) * 32;
  if (st == ST_F64)
    integral_partial_kernel<double><<<l.nblocks, threads, 0, stream>>>(
        l.V, static_cast<const double*>(l.x), l.count, l.chunk, l.nlev, l.ld, l.part);
  else if (st == ST_BF16)
    integral_partial_kernel<uint16_t><<<l.nblocks, threads, 0, stream>>>(
        l.V, static_cast<const uint16_t*>(l.x), l.count, l.chunk, l.nlev, l.ld, l.part);
  else
    integral_partial_kernel<float><<<l.nblocks, threads, 0, stream>>>(
        l.V, static_cast<const float*>(l.x), l.count, l.chunk, l.nlev, l.ld, l.part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  integral_final_kernel<<<(l.nlev + 255) / 256, 256, 0, stream>>>(l.part, l.nblocks, l.nlev, l.out);
  return cudaGetLastError();
}

cudaError_t launch_fp64_fma(double* out, int blocks, int threads, int64_t iters, cudaStream_t stream) {
  fp64_fma_kernel<<<blocks, threads, 0, stream>>>(out, iters);
  return cudaGetLastError();
}

cudaError_t launch_remap(StorageType st, const RemapLaunch& r, cudaStream_t stream) {
  return r.idx32 ? remap_st<true>(st, r, stream) : remap_st<false>(st, r, stream);
}

cudaError_t launch_batch(StorageType st, int vec, bool idx32, const BatchParams& params, int threads, int blocks,
                         cudaStream_t stream) {
  if (st != ST_F64 && st != ST_F32) return cudaErrorInvalidValue;
  void* args[] = {const_cast<BatchParams*>(&params)};
  return cudaLaunchKernel(batch_fn(st, vec, idx32), dim3(blocks), dim3(threads), args, 0, stream);
}

int batch_occupancy(StorageType st, int vec, bool idx32, int threads) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_fn(st, vec, idx32), threads, 0) != cudaSuccess)
    return 1;
  return blocks > 0 ? blocks : 1;
}

}  // namespace atlasgb
