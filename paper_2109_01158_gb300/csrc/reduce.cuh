// reduce.cuh -- fixed-order multi-value sums over a grid, finished by the last block.
//
// Each block sums NV values per thread in a fixed tree (warp shuffles, then one warp over
// the per-warp totals) and writes them to part[block * NV + j]; the block that takes the last
// ticket sums the partials in block order and resets the ticket.  The grid of the callers
// depends only on the vector length, so the results are bitwise reproducible.
#pragma once

#include "fe_internal.cuh"

namespace fe {
namespace {

__device__ __forceinline__ double red_warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Block totals of NV values per thread; valid in thread 0.
template <int NV>
__device__ __forceinline__ void red_block_sum(double (&x)[NV]) {
  __shared__ double sh[NV > 0 ? NV : 1][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    x[j] = red_warp_sum(x[j]);
    if (lane == 0) sh[j][warp] = x[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    x[j] = (threadIdx.x < kThreads / 32) ? sh[j][threadIdx.x] : 0.0;
    if (warp == 0) x[j] = red_warp_sum(x[j]);
  }
}

// Grid totals: true in thread 0 of the block that finishes last, with the totals in tot.
template <int NV>
__device__ __forceinline__ bool red_finish(double (&acc)[NV], double* part, unsigned* ticket, double (&tot)[NV]) {
  __shared__ bool am_last;
  red_block_sum<NV>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[(int64_t)blockIdx.x * NV + j] = acc[j];
    __threadfence();
    am_last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads)
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] += __ldcg(part + (int64_t)b * NV + j);
  red_block_sum<NV>(tot);
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

}  // namespace
}  // namespace fe
