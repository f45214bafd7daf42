// tile_common.cuh -- pieces shared by the fused element + patch kernels of every precision
// (see fe_tiles.cu for the tile structure): the shared-memory layout of the tile pipeline, the
// asynchronous copies that fill it, the per-tile energy partials and their final sum, and the
// kernel that completes the gradient of the shared nodes.
//
// The fused kernels run one persistent block per SM; block b takes the tiles b, b + G,
// b + 2G, ... (G blocks).  Its warps are specialised: element warps (one thread per element of
// a tile), node warps (the nodal values of the next tile, then the patch sums of the current
// one) and a producer warp (bulk asynchronous copies (TMA) of the element arrays and node
// records of the following tiles, and the tiles' energy partials).  They hand buffers to each
// other through full/empty mbarriers, so the element arithmetic of one tile overlaps the patch
// sums of the previous one and the HBM traffic of the next ones.
#pragma once

#include "async_copy.cuh"
#include "df64.cuh"
#include "fe_internal.cuh"

namespace fe {
namespace {

// float -> double from the bits (exact, like the conversion instruction, which runs at a low
// rate on the FP64 unit of this GPU): sign, exponent rebiased by 1023 - 127, significand
// shifted up by 29.  Zero, subnormals, Inf and NaN take the conversion instruction.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)f;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu)), (int)(u << 29));
}

// Shared-memory layout of the pipeline of one block (buffers of consecutive tiles alternate):
//   E[2]   element stages: DIM*DIM shape-gradient arrays and the volume (EB bytes per element
//          each), then the local ids / local slots (16 bytes per element): the layout of a
//          tile's block in device memory, which one bulk copy stages;
//   R[kRecBufs]  node records (int4 per tile node);
//   U[2]   the tile's nodal values, NU bytes per node;
//   Rs[2]  the tile's local forces: D columns (one per component) of RB bytes per slot,
//          each column 16 bytes longer than the slots (so the columns of one slot fall in
//          different shared-memory banks);
//   Ew[2]  the tile's energy |T| W per element warp (a float each);
//   Bd[kRecBufs]  the tile nodes' load b_i (D doubles per node) and Dirichlet mask (an int per
//          node, bit j for dof j), copied by the node warps with the nodal values, so that the
//          patch sums read them from shared memory; as many buffers as the records, as they
//          are read until the patch sums of the tile are done.
// The records are requested kRecBufs tiles ahead, so that their copies are never what the
// gather of a tile's nodal values waits for.
constexpr int kRecBufs = 4;

template <int DIM, int D, int EB, int NU, int RB>
struct TilePipe {
  static constexpr int kNodes = tile_max_nodes(DIM);
  static constexpr int kSlots = (DIM + 1) * kTileElems;
  static constexpr int kArrays = DIM * DIM + 1;
  static constexpr int kArrayBytes = (kTileElems * EB + 15) / 16 * 16;
  static_assert(kTileElems % kTileAlign == 0, "tiles hold whole groups of kTileAlign elements");
  static constexpr int kElemOff = kArrays * kArrayBytes;          // uint4 per element
  static constexpr int kEBytes = kElemOff + kTileElems * 16;
  static constexpr int kRBytes = kNodes * 16;
  static constexpr int kUBytes = (kNodes * NU + 15) / 16 * 16;
  static constexpr int kColBytes = (kSlots * RB + 15) / 16 * 16 + 16;   // one component's column
  static constexpr int kRsBytes = D * kColBytes;
  static constexpr int kEwBytes = (kTileElems / 32 * 4 + 15) / 16 * 16;
  static constexpr int kBdMaskOff = kNodes * D * 8;                 // ints after the doubles
  static constexpr int kBdBytes = (kBdMaskOff + kNodes * 4 + 15) / 16 * 16;
  static constexpr int kE = 0;
  static constexpr int kR = kE + 2 * kEBytes;
  static constexpr int kU = kR + kRecBufs * kRBytes;
  static constexpr int kRs = kU + 2 * kUBytes;
  static constexpr int kEw = kRs + 2 * kRsBytes;
  static constexpr int kBd = kEw + 2 * kEwBytes;
  static constexpr int kBytes = kBd + kRecBufs * kBdBytes;
  // (the kernels also hold about 300 bytes of static shared memory: barriers and tile info)
  static_assert(kBytes + 512 <= 227 * 1024, "the pipeline must fit in the shared memory of one block");
  static_assert(kEBytes % 16 == 0 && kRBytes % 16 == 0, "alignment");
  static_assert(2 * kRsBytes >= 2 * kTileThreads * 8, "the final reduction reuses Rs");
};

// The tile structure and element blocks of one precision.
struct TileArgs {
  const int32_t* ebeg;         // ntiles + 1
  const int32_t* nbeg;         // ntiles + 1
  const int4* node;            // node records
  const unsigned char* blk;    // ntiles blocks of S::kEBytes: the layout of an element stage
  int64_t ntiles;
  int64_t npart;               // partial slots of the shared nodes
  long long wait_limit;
};

// Thread 0: one bulk copy of tile t's element block into the stage at `st`, completing on
// `bar` (one arrival and the block's bytes).  The stage was last read by ordinary loads of the
// element warps, which released it through the empty barrier the caller waited for; a bulk
// copy that overwrites data read that way needs no proxy fence (only data written by ordinary
// stores and read by the copy engine would).
template <class S>
__device__ __forceinline__ void pipe_issue_elems(unsigned char* st, const TileArgs& A, int64_t t, uint64_t* bar) {
  mbar_arrive_expect_tx(bar, (uint32_t)S::kEBytes);
  bulk_g2s(st, A.blk + t * S::kEBytes, (uint32_t)S::kEBytes, bar);
}

// Thread 0: bulk copy of the node records [k0, k0 + nt) into `rb`, completing on `bar` (the
// slot was released like an element stage, so no proxy fence either).
__device__ __forceinline__ void pipe_issue_recs(int4* rb, const TileArgs& A, int k0, int nt, uint64_t* bar) {
  mbar_arrive_expect_tx(bar, (uint32_t)nt * 16u);
  if (nt > 0) bulk_g2s(rb, A.node + k0, (uint32_t)nt * 16u, bar);
}

__device__ __forceinline__ double pipe_warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ void pipe_warp_pair_sum(const double* r0, const double* r1, int n, double* s0,
                                                   double* s1) {
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
  for (int k = lane; k < n; k += 32) {
    a += r0[k];
    b += r1[k];
  }
  *s0 = pipe_warp_sum(a);
  *s1 = pipe_warp_sum(b);
}

// After every block has written its tiles' partials epart[t] (sum |T| W) and fenced them: the
// block that arrives last adds them over the tiles in a fixed order, and the node-side b.v
// partials bvp[0 .. nbv) likewise, and writes J = sum |T| W - (b.v + shift) (shift = b.X
// when the caller passes displacements).  `red` holds 2 * blockDim.x doubles.
__device__ __forceinline__ void pipe_finish_energy(const double* epart, int64_t ntiles, const double* bvp, int nbv,
                                                   double shift, unsigned* counter, double* J, double* red) {
  __shared__ bool am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(counter, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double s = 0.0, b = 0.0;
  for (int64_t k = threadIdx.x; k < ntiles; k += blockDim.x) s += __ldcg(epart + k);
  if (bvp)
    for (int k = threadIdx.x; k < nbv; k += blockDim.x) b += __ldcg(bvp + k);
  red[threadIdx.x] = s;
  red[blockDim.x + threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double ts, tb;
    pipe_warp_pair_sum(red, red + blockDim.x, blockDim.x, &ts, &tb);
    if (threadIdx.x == 0) {
      *J = ts - (tb + shift);
      *counter = 0u;
    }
  }
}

// Accumulator of a shared node's partial sums (one per tile, in tile order).
struct PartF32 {
  using T = float;
  float s = 0.f;
  __device__ __forceinline__ void add(float x, bool first) { s = first ? x : __fadd_rn(s, x); }
  __device__ __forceinline__ double value() const { return f2d_bits(s); }
};

struct PartDF {
  using T = float2;
  df s = {0.f, 0.f};
  __device__ __forceinline__ void add(float2 x, bool first) { s = first ? df{x.x, x.y} : df_add(s, df{x.x, x.y}); }
  __device__ __forceinline__ double value() const { return df_to_double(s); }
};

// Gradient of the shared nodes: g_i = sum of the node's tile partials - b_i, 0 on Dirichlet
// dofs; written at the caller's index perm[i] (perm null = identity).  One thread per
// (node, component).
template <int D, class Acc>
__global__ void __launch_bounds__(kThreads) k_tile_shared(int64_t nshared, const int32_t* __restrict__ snode,
                                                          const int32_t* __restrict__ sbeg,
                                                          const int32_t* __restrict__ spart,
                                                          const typename Acc::T* __restrict__ part,
                                                          const double* __restrict__ b,
                                                          const uint8_t* __restrict__ dir,
                                                          const int32_t* __restrict__ perm, double* __restrict__ g) {
  const int64_t n = nshared * D;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += stride) {
    const int64_t s = w / D;
    const int j = (int)(w - s * D);
    const int64_t i = __ldg(snode + s);
    const int32_t p0 = __ldg(sbeg + s), p1 = __ldg(sbeg + s + 1);
    Acc acc;
    for (int32_t p = p0; p < p1; ++p) acc.add(__ldg(part + (int64_t)__ldg(spart + p) * D + j), p == p0);
    const int64_t dst = perm ? (int64_t)__ldg(perm + i) : i;
    g[dst * D + j] = __ldg(dir + i * D + j) ? 0.0 : (b ? acc.value() - __ldg(b + i * D + j) : acc.value());
  }
}

}  // namespace
}  // namespace fe
