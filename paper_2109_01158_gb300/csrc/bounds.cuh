// bounds.cuh -- device index checks of the bounds-checking build (not in the paper).
//
// Built with -DFE_DEBUG_BOUNDS (build.build(bounds=True): libfemenergy_bounds.so), every index
// a kernel reads from memory and then uses to address another buffer goes through FE_CHK: an
// index outside [0, n) is not used (the access takes index 0 instead, which is in bounds for
// every checked buffer, as none of them is empty when a thread reaches it), and the first such
// index is recorded in an error word together with the site that saw it.  The kernel never
// traps: the call completes, its results are wrong, and fe_debug_bounds() on the host reads
// and clears the record.  In the ordinary build FE_CHK is the index itself and nothing of this
// file is compiled in.
//
// Every translation unit that includes this header has its own error word (a __device__
// variable is per unit without relocatable device code); each unit registers a reader of its
// word with the library at load time, and fe_debug_bounds() asks them all.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fe {

// Sites of the checks (the record keeps the first one seen).
enum BoundsSite : int {
  kSiteNodePerm = 1,      // node preparation: caller index perm[i] < nn
  kSiteElemNode = 2,      // element kernels: node id of an element < nn
  kSiteElemSlot = 3,      // element kernels: CSR slot of (element, local node) < ne (dim + 1)
  kSiteElemPerm = 4,      // element kernels: caller element index eperm[e] < ne
  kSiteGatherPerm = 5,    // patch gather: caller index perm[i] < nn
  kSiteGatherRow = 6,     // patch gather: a node's CSR row inside its warp's staged range
  kSiteTileNode = 7,      // FP32 tiles: node id of a tile record < nn
  kSiteTileLocal = 8,     // FP32 tiles: local node id of an element < the tile's node count
  kSiteTileSlot = 9,      // FP32 tiles: local slot of (element, local node) < slots of a tile
  kSiteTilePart = 10,     // FP32 tiles: partial slot of a shared node < partial slots
  kSiteSelfTest = 99,     // fe_debug_bounds_selftest
};

#ifdef FE_DEBUG_BOUNDS

// Registry of the per-unit readers (fe_api.cu): read the unit's word on the current device
// and clear it.
using BoundsReader = cudaError_t (*)(unsigned long long* word);
void register_bounds_reader(BoundsReader f);

namespace {

__device__ unsigned long long g_bounds_word;   // (site << 48) | low 48 bits of the index

__device__ __forceinline__ int64_t bounds_check(int64_t i, int64_t n, int site) {
  if ((uint64_t)i < (uint64_t)n) return i;
  const unsigned long long w = ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffULL);
  atomicCAS(&g_bounds_word, 0ULL, w);
  return 0;
}

cudaError_t bounds_read_clear(unsigned long long* word) {
  cudaError_t e = cudaMemcpyFromSymbol(word, g_bounds_word, sizeof(*word));
  if (e != cudaSuccess) return e;
  const unsigned long long zero = 0;
  return cudaMemcpyToSymbol(g_bounds_word, &zero, sizeof(zero));
}

struct BoundsRegistrar {
  BoundsRegistrar() { register_bounds_reader(&bounds_read_clear); }
};
const BoundsRegistrar g_bounds_registrar;

}  // namespace

#define FE_CHK(i, n, site) ::fe::bounds_check((int64_t)(i), (int64_t)(n), (site))

#else

#define FE_CHK(i, n, site) (i)

#endif

}  // namespace fe
