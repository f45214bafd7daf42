// tile_stream.cuh -- streaming of element tiles into shared memory with bulk (TMA) copies.
//
// An element kernel reads, per element, one entry of each of several structure-of-arrays
// streams (shape gradients, volume, node ids, CSR slots).  Instead of one global load per
// entry and thread, a block owns tiles of kTile consecutive elements; for each tile one
// thread issues one cp.async.bulk per array into a shared-memory stage, and a ring of
// kStages stages keeps the next tiles in flight while the current one is computed.
//
// An array whose start is not 16-byte aligned is copied from the aligned address below it;
// its constant offset (`shift`) is added when an entry is read back from shared memory.
#pragma once

#include "async_copy.cuh"
#include "fe_internal.cuh"

namespace fe {

constexpr int kTile = 32;                             // elements per tile = threads per block
constexpr int kStages = 3;
constexpr int kTileMinBlocks = 20 * 32 / kTile;       // blocks per SM asked of the compiler: 20 warps
constexpr int kTileBlocks = 152 * (512 / kTile);      // fixed persistent grid: 512 threads on each of 152 SMs

template <int NARR>
struct TileArrays {
  const unsigned char* base[NARR];  // start of each array (entry 0)
  int esize[NARR];                   // bytes per entry (4 or 8)
};

// Shared-memory layout of one stage for the arrays of `A`.
template <int NARR>
struct TileLayout {
  int off[NARR];
  int shift[NARR];
  int stage_bytes;
  __device__ __forceinline__ void init(const TileArrays<NARR>& A) {
    int o = 0;
#pragma unroll
    for (int a = 0; a < NARR; ++a) {
      off[a] = o;
      shift[a] = (int)(reinterpret_cast<uintptr_t>(A.base[a]) & 15u);
      o += ((kTile * A.esize[a] + 16) + 15) & ~15;
    }
    stage_bytes = o;
  }
};

// Thread-0 side: copy tile `tile` (elements tile*kTile .. min(+kTile, ne)) of every array
// into `stage`, completing on `bar`.
template <int NARR>
__device__ __forceinline__ void tile_issue(const TileArrays<NARR>& A, const TileLayout<NARR>& L,
                                           unsigned char* stage, uint64_t* bar, int64_t tile, int64_t ne) {
  const int64_t first = tile * kTile;
  const int n = (int)((ne - first) < kTile ? (ne - first) : kTile);
  uint32_t total = 0;
  uint32_t bytes[NARR];
#pragma unroll
  for (int a = 0; a < NARR; ++a) {
    bytes[a] = (uint32_t)((L.shift[a] + n * A.esize[a] + 15) & ~15);
    total += bytes[a];
  }
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, total);
#pragma unroll
  for (int a = 0; a < NARR; ++a) {
    const unsigned char* src = A.base[a] + first * A.esize[a] - L.shift[a];
    bulk_g2s(stage + L.off[a], src, bytes[a], bar);
  }
}

template <typename T, int NARR>
__device__ __forceinline__ T tile_get(const unsigned char* stage, const TileLayout<NARR>& L, int a, int e,
                                      int esize) {
  return *reinterpret_cast<const T*>(stage + L.off[a] + L.shift[a] + e * esize);
}

}  // namespace fe
