// fe_eval_f32.cu -- the FP32 path (FE_F32_COMP; a precision variant not in the paper): the
// energy J(v) = sum |T| W(F_T) - b.v and its exact gradient (Sec. 5 and 6.2) with the element
// arithmetic in float (elem_f32.cuh) and FP64 energy sums.
//
// Three launches per call:
//   k_pairs32     one thread per node: u = v - X in FP64 (v in the caller's or the device
//                 numbering; u = v for the p-Laplacian or a displacement input), stored as
//                 float pairs (hi, lo) so that differences across an element round only once,
//                 and the block partials of b.v;
//   k_tile_f32    one persistent block per SM walks its element tiles (fe_tiles.cu,
//                 tile_common.cuh) with specialised warps:
//                   the producer warp stages each tile's element block (dphi, vol, local
//                      ids and slots, laid out per tile by k_tile_blocks32) with one bulk
//                      copy, and its node records with another;
//                   node warps copy the tile's float pairs, b_i and Dirichlet masks into
//                      shared memory;
//                   element warps, one thread per element: H from float-pair differences of
//                      u, W and |T| dW/dF in float, and the local forces
//                      r_{T,l} = |T| dW/dF grad(phi_l) written to the element's local slots in
//                      shared memory; then the patch sums of the previous tile, one thread per
//                      (tile node, component): the node's local slots summed in float in a
//                      fixed order; a node whose patch lies in the tile gets g_i = sum - b_i
//                      (0 on Dirichlet dofs), a shared node leaves its partial sum;
//                   each element warp adds its |T| W by a pairwise tree in float, and the
//                      producer the tile's warp sums by a TwoSum tree (float pairs) into the
//                      tile's energy partial (FP64); the last block adds the partials in tile
//                      order;
//   k_tile_shared adds the shared nodes' partials in tile order.
// The local forces never leave the chip (only the shared nodes' partials do), and every sum
// has a fixed order: bitwise reproducible whatever the number of blocks.
#include "elem_f32.cuh"
#include "fe_internal.cuh"
#include "tile_common.cuh"

namespace fe {
namespace {

template <int DIM, int D>
struct Pipe32 {
  static constexpr int DP = D == 3 ? 4 : D;   // float pairs per node record (padded)
  // nodal values: DP float pairs per node; r: one float column per component
  using S = TilePipe<DIM, D, 4, DP * 8, 4>;
};

template <int D>
__device__ __forceinline__ void load_pairs_g(const float2* __restrict__ u, int64_t n, float2 (&w)[D]) {
  if constexpr (D == 1) {
    w[0] = __ldg(u + n);
  } else if constexpr (D == 2) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(u) + n);
    w[0] = make_float2(a.x, a.y);
    w[1] = make_float2(a.z, a.w);
  } else {
    const float4* p = reinterpret_cast<const float4*>(u) + 2 * n;
    const float4 a = __ldg(p), b = __ldg(p + 1);
    w[0] = make_float2(a.x, a.y);
    w[1] = make_float2(a.z, a.w);
    w[2] = make_float2(b.x, b.y);
  }
}

// The D float pairs of tile node k from shared memory (DP pairs per node).
template <int D, int DP>
__device__ __forceinline__ void load_pairs_s(const float2* us, int k, float2 (&w)[D]) {
  if constexpr (DP == 1) {
    w[0] = us[k];
  } else if constexpr (DP == 2) {
    const float4 a = reinterpret_cast<const float4*>(us)[k];
    w[0] = make_float2(a.x, a.y);
    w[1] = make_float2(a.z, a.w);
  } else {
    const float4* p = reinterpret_cast<const float4*>(us) + 2 * k;
    const float4 a = p[0], b = p[1];
    w[0] = make_float2(a.x, a.y);
    w[1] = make_float2(a.z, a.w);
    w[2] = make_float2(b.x, b.y);
  }
}

// d as the pair hi + lo of floats: hi = d with its significand cut to 24 bits, lo = the rest
// cut to 24 bits (|hi + lo - d| < 2^-47 |d|), from the bits of d with integer operations only
// (the conversion instructions run at a low rate on the FP64 unit of this GPU).  Outside
// 2^-60 <= |d| < 2^61 (and for 0, subnormals, Inf, NaN) it rounds in FP64.
__device__ __forceinline__ float2 split_double(double d) {
  const long long bits = __double_as_longlong(d);
  const unsigned hw = (unsigned)(bits >> 32);
  const unsigned ex = (hw >> 20) & 0x7ffu;
  if (ex - (1023u - 60u) >= 121u) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
  }
  const unsigned sign = hw & 0x80000000u;
  // hi: sign | float exponent | the top 23 stored significand bits
  const float hi = __uint_as_float(sign | ((ex - 896u) << 23) | ((unsigned)(bits >> 29) & 0x7fffffu));
  // lo: the low 29 significand bits, worth rest * 2^(ex - 1075), normalised to a float with
  // its top 24 bits (nb significant bits: exponent nb - 1 + ex - 1075, at least 2^-112)
  const unsigned rest = (unsigned)bits & 0x1fffffffu;
  if (rest == 0u) return make_float2(hi, 0.f);
  const int nb = 32 - __clz(rest);
  const unsigned m = nb > 24 ? rest >> (nb - 24) : rest << (24 - nb);
  const float lo = __uint_as_float(sign | ((unsigned)(nb + (int)ex - 949) << 23) | (m & 0x7fffffu));
  return make_float2(hi, lo);
}

// u (device order) as float pairs, DP pairs per node, one node per thread; block partials of
// b.v (b in device order, v read at the caller's index when perm is given; the grid depends on
// nn only, so the partials are the same on every run).
template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_pairs32(int64_t nn, const double* __restrict__ v,
                                                      const double* __restrict__ X, const int32_t* __restrict__ perm,
                                                      const double* __restrict__ b, float2* __restrict__ u, bool disp,
                                                      double* __restrict__ bv_partials) {
  constexpr int DP = Pipe32<DIM, D>::DP;
  __shared__ double sh[kThreads / 32];
  double dot = 0.0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // one node per thread
  if (i < nn) {
    const int64_t src = perm ? (int64_t)FE_CHK(__ldg(perm + i), nn, kSiteNodePerm) : i;
    float2 w[DP];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const double vj = __ldg(v + src * D + j);
      w[j] = split_double((MODEL == FE_NEOHOOKE && !disp) ? vj - __ldg(X + i * DIM + j) : vj);
      if (b) dot = fma(__ldg(b + i * D + j), vj, dot);
    }
    if constexpr (DP == 1) {
      u[i] = w[0];
    } else if constexpr (DP == 2) {
      reinterpret_cast<float4*>(u)[i] = make_float4(w[0].x, w[0].y, w[1].x, w[1].y);
    } else {
      float4* o = reinterpret_cast<float4*>(u) + 2 * i;
      o[0] = make_float4(w[0].x, w[0].y, w[1].x, w[1].y);
      o[1] = make_float4(w[2].x, w[2].y, 0.f, 0.f);
    }
  }
  if (b) {
    // a fixed tree per block (the grid depends on nn only)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x < 32) {
      dot = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
      if (threadIdx.x == 0) bv_partials[blockIdx.x] = dot;
    }
  }
}

// Barriers of the tile pipeline (index: buffer of the tile).
struct PipeBars {
  uint64_t e_full[2];                // element stage: its bulk copy landed
  uint64_t in_full[2];               // element stage landed and nodal values written
  uint64_t in_empty[2];              // element warps done with the element stage and nodal values
  uint64_t r_full[kRecBufs], r_empty[kRecBufs];   // node records: landed / patch sums done
  uint64_t rs_full[2], rs_empty[2];  // local forces and energies: element warps wrote / patch
                                     // sums and producer done
};

// The block: warps 0 .. kTileElems/32 - 1 are element warps (one thread per element of a
// tile); the next kTileNodeWarps are node warps (they copy the next tile's nodal values into
// shared memory, then sum the current tile's patches); the last warp is the producer (its lane
// 0 issues every bulk copy; the warp adds each tile's energy partial).  The roles hand buffers
// over through the mbarriers of PipeBars; every wait is bounded and gives up when another
// thread has given up, so a lost copy ends the kernel with FE_ETIMEOUT instead of a hang.
template <int DIM, int D, int MODEL, bool ENERGY, bool GRAD, bool DENS>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile_f32(
    TileArgs ta, const float2* __restrict__ upairs, const double* __restrict__ b, const uint8_t* __restrict__ dir,
    const int32_t* __restrict__ eperm, ModelParams mp, bool caller_order, double* __restrict__ g,
    float* __restrict__ part, double* __restrict__ dens, double* epart, const double* bvp, int nbv, double shift,
    unsigned* counter, double* J, int* status) {
  using P = Pipe32<DIM, D>;
  using S = typename P::S;
  constexpr int K = DIM + 1, DP = P::DP;
  constexpr int NE = kTileElems, NEW = NE / 32;              // element threads and warps
  static_assert(NEW <= 32, "the producer adds one energy pair per element warp in one warp");
  constexpr int NN = 32 * kTileNodeWarps;                    // node threads
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ PipeBars bars;
  __shared__ int4 info[kRecBufs];        // {e0, e1, k0, nt} of the tile whose records are in R[slot]
  __shared__ volatile int abort_flag;
  const int G = gridDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool elem_warp = warp < NEW, node_warp = !elem_warp && warp < NEW + kTileNodeWarps;
  const bool issuer = tid == NE + NN;
  const int64_t ntiles = ta.ntiles;
  const int my_tiles = (int)((ntiles - blockIdx.x + G - 1) / G);   // tiles blockIdx.x + i G
  auto tile_of = [&](int i) { return (int64_t)blockIdx.x + (int64_t)i * G; };
  auto E = [&](int i) { return smem + S::kE + (i & 1) * S::kEBytes; };
  auto R = [&](int i) { return reinterpret_cast<int4*>(smem + S::kR + (i % kRecBufs) * S::kRBytes); };
  auto U = [&](int i) { return reinterpret_cast<float2*>(smem + S::kU + (i & 1) * S::kUBytes); };
  // component j of the local forces of tile i, by local slot
  auto RC = [&](int i, int j) { return reinterpret_cast<float*>(smem + S::kRs + (i & 1) * S::kRsBytes + j * S::kColBytes); };
  auto EW = [&](int i) { return reinterpret_cast<float*>(smem + S::kEw + (i & 1) * S::kEwBytes); };
  auto BDB = [&](int i) { return reinterpret_cast<double*>(smem + S::kBd + (i % kRecBufs) * S::kBdBytes); };
  auto BDM = [&](int i) { return reinterpret_cast<int*>(smem + S::kBd + (i % kRecBufs) * S::kBdBytes + S::kBdMaskOff); };
  // every thread of a warp calls wait() together and gets the same answer (the warp leaves the
  // pipeline as a whole, so no lane is left behind in a warp-wide operation)
  bool ok = true;
  auto wait = [&](uint64_t* bar, int use) {   // the use-th completion of `bar`
    bool w = ok && mbar_wait_or_abort(bar, (uint32_t)use & 1u, ta.wait_limit, &abort_flag);
    if (ok && !w && !abort_flag) {
      abort_flag = 1;
      atomicOr(status, kStatusTimeout);
    }
    ok = __all_sync(0xffffffffu, w);
    return ok;
  };
  // the same for a wait done by lane 0 alone (the result is broadcast to the warp)
  auto wait_lane0 = [&](uint64_t* bar, int use) {
    bool w = true;
    if (lane == 0) {
      w = ok && mbar_wait_or_abort(bar, (uint32_t)use & 1u, ta.wait_limit, &abort_flag);
      if (ok && !w && !abort_flag) {
        abort_flag = 1;
        atomicOr(status, kStatusTimeout);
      }
    }
    ok = __shfl_sync(0xffffffffu, w, 0) && ok;
    return ok;
  };
  // the issuer's copies: how many were issued into each buffer (to drain them on abort)
  int nE[2] = {0, 0}, nR[kRecBufs] = {};
  auto issue_elems = [&](int i) {
    pipe_issue_elems<S>(E(i), ta, tile_of(i), &bars.e_full[i & 1]);
    ++nE[i & 1];
  };
  // the element and node ranges of the next tile whose records are issued, loaded one issue
  // ahead so that the issuer does not wait for them
  int4 pre = make_int4(0, 0, 0, 0);
  int pre_i = -1;
  auto load_pre = [&](int i) {
    if (i >= my_tiles) return;
    const int64_t tq = tile_of(i);
    pre = make_int4(__ldg(ta.ebeg + tq), __ldg(ta.ebeg + tq + 1), __ldg(ta.nbeg + tq), __ldg(ta.nbeg + tq + 1));
    pre_i = i;
  };
  auto issue_recs = [&](int i) {
    if (pre_i != i) load_pre(i);
    const int4 raw = pre;
    info[i % kRecBufs] = make_int4(raw.x, raw.y, raw.z, raw.w - raw.z);
    pipe_issue_recs(R(i), ta, raw.z, raw.w - raw.z, &bars.r_full[i % kRecBufs]);
    ++nR[i % kRecBufs];
    load_pre(i + 1);
  };
  if (tid == 0) abort_flag = 0;
  if (issuer) {
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bars.e_full[q], 1);
      mbar_init(&bars.in_full[q], kTileNodeWarps);
      mbar_init(&bars.in_empty[q], NEW);
      mbar_init(&bars.rs_full[q], NEW);
      mbar_init(&bars.rs_empty[q], NEW + 1);
    }
    for (int q = 0; q < kRecBufs; ++q) {
      mbar_init(&bars.r_full[q], 1);
      mbar_init(&bars.r_empty[q], NEW);
    }
    mbar_init_fence();
  }
  __syncthreads();

  bool bad = false;
  if (warp == NEW + kTileNodeWarps) {
    // producer warp: lane 0 issues the bulk copies; the warp adds the tiles' energy partials
    if (issuer) {
      // records of the first kRecBufs tiles, elements of the first two
      for (int i = 0; i < kRecBufs && i < my_tiles; ++i) issue_recs(i);
      for (int i = 0; i < 2 && i < my_tiles; ++i) issue_elems(i);
    }
    // In the order the element warps free the buffers: the element stage of tile i when they
    // are done with its elements (B(i)), which is also when its energies are complete; the
    // record slot of tile i - 1 only after its patch sums (C(i - 1), done after B(i)), so that
    // the next element copy never waits behind patch sums.
    for (int i = 0; i < my_tiles; ++i) {
      if (i + 2 < my_tiles) {
        if (!wait_lane0(&bars.in_empty[i & 1], i >> 1)) break;
        if (issuer) issue_elems(i + 2);
      }
      if (!wait(&bars.rs_full[i & 1], i >> 1)) break;
      if (ENERGY) {
        // the element warps' sums as float pairs, added by a fixed TwoSum tree across the lanes
        // (FP32 operations: a chain of FP64 additions has a long latency on this GPU), then
        // hi + lo in FP64; +Inf apart, as TwoSum on Inf gives NaN
        const float w = lane < NEW ? EW(i)[lane] : 0.f;
        const bool inf = __any_sync(0xffffffffu, isinf(w));
        df p = {isinf(w) ? 0.f : w, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const df q = {__shfl_down_sync(0xffffffffu, p.hi, o), __shfl_down_sync(0xffffffffu, p.lo, o)};
          p = df_add(p, q);
        }
        if (lane == 0) epart[tile_of(i)] = inf ? CUDART_INF : f2d_bits(p.hi) + f2d_bits(p.lo);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.rs_empty[i & 1]);
      if (i >= 1 && i - 1 + kRecBufs < my_tiles) {
        if (!wait_lane0(&bars.r_empty[(i - 1) % kRecBufs], (i - 1) / kRecBufs)) break;
        if (issuer) issue_recs(i - 1 + kRecBufs);
      }
    }
  } else if (node_warp) {
    const int ntid = tid - NE;
    // the nodal values of tile i (its records must have landed) into U(i)
    auto gather = [&](int i) {
      if (!wait(&bars.r_full[i % kRecBufs], i / kRecBufs)) return false;
      if (i >= 2 && !wait(&bars.in_empty[i & 1], (i >> 1) - 1)) return false;
      const int4* rec = R(i);
      float2* us = U(i);
      const int nt = info[i % kRecBufs].w;
      double* bd = BDB(i);
      int* bm = BDM(i);
      // all loads of a thread's nodes first, then the stores: the loads are in flight together
      // instead of one round trip per node; with the nodal values, each node's load b_i and
      // Dirichlet mask for the patch sums
      constexpr int RN = (S::kNodes + NN - 1) / NN;
      float2 w[RN][D];
      double bb[RN][D];
      int mk[RN];
#pragma unroll
      for (int q = 0; q < RN; ++q) {
        const int k = ntid + q * NN;
        mk[q] = 0;
        if (k < nt) {
          const int64_t n = FE_CHK(rec[k].x, mp.nn, kSiteTileNode);
          load_pairs_g<D>(upairs, n, w[q]);
#pragma unroll
          for (int j = 0; j < D; ++j) {
            bb[q][j] = (GRAD && b) ? __ldg(b + n * D + j) : 0.0;
            if (GRAD) mk[q] |= __ldg(dir + n * D + j) ? (1 << j) : 0;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RN; ++q) {
        const int k = ntid + q * NN;
        if (k < nt) {
#pragma unroll
          for (int j = 0; j < D; ++j) {
            us[k * DP + j] = w[q][j];
            if (GRAD) bd[k * D + j] = bb[q][j];
          }
          if (GRAD) bm[k] = mk[q];
        }
      }
      // the first node warp also waits for the tile's element copy, so that the element warps
      // wait on one barrier for both (its completion orders the copy before their loads)
      if (warp == NEW && !wait(&bars.e_full[i & 1], i >> 1)) return false;
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.in_full[i & 1]);
      return true;
    };
    if (my_tiles > 0) gather(0);
    for (int i = 1; i < my_tiles && ok; ++i)
      if (!gather(i)) break;
  } else if (elem_warp) {
    // Software-pipelined over the tiles: B (the elements) of tile i, then C (the patch sums)
    // of tile i - 1, whose forces every element warp wrote before its own B of tile i -- so a
    // warp that finishes B early goes on to C instead of waiting for the slowest warp.
    const float C1 = (float)mp.C1, D1 = (float)mp.D1;
    // C: the patch sums of tile i, one thread per (tile node, component)
    auto patch_sums = [&](int i) {
      if (!wait(&bars.rs_full[i & 1], i >> 1)) return false;
      if (GRAD) {
        const int4* Rr = R(i);
        const float* rc0 = RC(i, 0);
        const double* bd = BDB(i);
        const int* bm = BDM(i);
        const int nt = info[i % kRecBufs].w;
        for (int w = tid; w < nt * D; w += NE) {
          const int k = w / D, j = w - k * D;
          const int4 rec = Rr[k];
          const int beg = rec.z & 0xffff, cnt = (int)((unsigned)rec.z >> 16);
          // the node's slots (consecutive in its column), two at a time: a first slot at an odd
          // position alone, then 8-byte pairs into two running sums (one paired addition per
          // pair), then a last odd slot; added in that fixed order
          const float* col = rc0 + j * (S::kColBytes / 4) + beg;
          float sum = 0.f;
          if (cnt > 0) {
            const int q0 = beg & 1;   // the column starts 16-byte aligned
            const float head = q0 ? col[0] : 0.f;
            const int np = (cnt - q0) >> 1;
            const float2* p2 = reinterpret_cast<const float2*>(col + q0);
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int t = 0; t < np; ++t) acc = __fadd2_rn(acc, p2[t]);
            const int qt = q0 + 2 * np;
            const float tail = qt < cnt ? col[qt] : 0.f;
            sum = __fadd_rn(__fadd_rn(__fadd_rn(head, acc.x), acc.y), tail);
          }
          const int dst = (rec.w >> 1) - 1;
          const int64_t n = FE_CHK(rec.x, mp.nn, kSiteTileNode);
          if (dst < 0) {
            const int64_t o = caller_order ? (int64_t)FE_CHK(rec.y, mp.nn, kSiteTileNode) : n;
            g[o * D + j] = ((bm[k] >> j) & 1) ? 0.0 : f2d_bits(sum) - bd[k * D + j];
          } else {
            part[(int64_t)FE_CHK(dst, ta.npart, kSiteTilePart) * D + j] = sum;
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars.rs_empty[i & 1]);
        mbar_arrive(&bars.r_empty[i % kRecBufs]);
      }
      return true;
    };
    for (int i = 0; i < my_tiles && ok; ++i) {
      // B: one thread per element of tile i
      if (!wait(&bars.in_full[i & 1], i >> 1)) break;
      if (i >= 2 && !wait(&bars.rs_empty[i & 1], (i >> 1) - 1)) break;
      const int4 in = info[i % kRecBufs];
      const unsigned char* St = E(i);
      const float2* us = U(i);
      float* rc0 = RC(i, 0);
      float ew = 0.f;
      const int e = in.x + tid;
      if (e < in.y) {
        const uint4 le = reinterpret_cast<const uint4*>(St + S::kElemOff)[tid];
        const int nt_i = in.w;
        const int lid[4] = {(int)FE_CHK(le.x & 0xffffu, nt_i, kSiteTileLocal), (int)FE_CHK(le.x >> 16, nt_i, kSiteTileLocal),
                            (int)FE_CHK(le.y & 0xffffu, nt_i, kSiteTileLocal), (int)FE_CHK(le.y >> 16, nt_i, kSiteTileLocal)};
        // each node's pairs in 16-byte loads (a node record is DP pairs, 16-byte aligned)
        float2 un[K][D];
#pragma unroll
        for (int l = 0; l < K; ++l) load_pairs_s<D, DP>(us, lid[l], un[l]);
        float a[DIM][D];
#pragma unroll
        for (int l = 1; l < K; ++l)
#pragma unroll
          for (int j = 0; j < D; ++j) a[l - 1][j] = pair_diff(un[l][j], un[0][j]);
        float gg[DIM][DIM];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
          for (int m = 0; m < DIM; ++m) gg[l][m] = reinterpret_cast<const float*>(St + (l * DIM + m) * S::kArrayBytes)[tid];
        const float vT = reinterpret_cast<const float*>(St + DIM * DIM * S::kArrayBytes)[tid];
        float Pm[D][DIM];
        const float W = elem_f32<DIM, D, MODEL, ENERGY || DENS, GRAD>(a, gg, vT, C1, D1, mp, Pm, bad);
        if (ENERGY) ew = __fmul_rn(vT, W);
        if (DENS) dens[eperm ? (int64_t)__ldg(eperm + e) : (int64_t)e] = (double)W;
        if (GRAD) {
          const int sl[4] = {(int)FE_CHK(le.z & 0xffffu, S::kSlots, kSiteTileSlot), (int)FE_CHK(le.z >> 16, S::kSlots, kSiteTileSlot),
                             (int)FE_CHK(le.w & 0xffffu, S::kSlots, kSiteTileSlot), (int)FE_CHK(le.w >> 16, S::kSlots, kSiteTileSlot)};
          float r0[D];
#pragma unroll
          for (int l = 1; l < K; ++l) {
            float r[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
              float s = __fmul_rn(Pm[j][0], gg[l - 1][0]);
#pragma unroll
              for (int m = 1; m < DIM; ++m) s = fmaf(Pm[j][m], gg[l - 1][m], s);
              r[j] = s;
              r0[j] = (l == 1) ? -s : __fsub_rn(r0[j], s);
            }
#pragma unroll
            for (int j = 0; j < D; ++j) rc0[j * (S::kColBytes / 4) + sl[l]] = r[j];
          }
#pragma unroll
          for (int j = 0; j < D; ++j) rc0[j * (S::kColBytes / 4) + sl[0]] = r0[j];
        }
      }
      if (ENERGY) {
        // the warp's |T| W by a fixed pairwise tree in float (every term >= 0, +Inf allowed:
        // relative error at most 5 roundings); the producer adds the tile's 24 warp sums
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ew = __fadd_rn(ew, __shfl_xor_sync(0xffffffffu, ew, o));
        if (lane == 0) EW(i)[warp] = ew;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars.in_empty[i & 1]);
        mbar_arrive(&bars.rs_full[i & 1]);
      }
      if (i >= 1 && !patch_sums(i - 1)) break;
    }
    if (ok && my_tiles > 0) patch_sums(my_tiles - 1);
  }

  __syncthreads();
  if (abort_flag) {
    // a wait gave up: wait with the full limit for every bulk copy still in flight (nothing may
    // land in shared memory after the block has left) and make J NaN
    if (issuer) {
      for (int q = 0; q < 2; ++q)
        if (nE[q] > 0) mbar_wait_bounded(&bars.e_full[q], (uint32_t)(nE[q] - 1) & 1u);
      for (int q = 0; q < kRecBufs; ++q)
        if (nR[q] > 0) mbar_wait_bounded(&bars.r_full[q], (uint32_t)(nR[q] - 1) & 1u);
      if (ENERGY)
        for (int i = 0; i < my_tiles; ++i) epart[tile_of(i)] = CUDART_NAN;
    }
  }
  if (ENERGY && warp == NEW + kTileNodeWarps && lane == 0) __threadfence();   // partials before the ticket
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) pipe_finish_energy(epart, ntiles, bvp, nbv, shift, counter, J, reinterpret_cast<double*>(smem + S::kRs));
}

// The tiles' element blocks: for tile t, its elements' dphi (DIM*DIM arrays) and vol in float,
// then their local ids / slots, each array at its offset of the element stage (S::kArrayBytes
// apart, S::kElemOff), element k of the tile at index k; entries past the tile's last element
// are zero.  One thread per (tile, element slot).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_tile_blocks32(int64_t ntiles, const int32_t* __restrict__ ebeg,
                                                            const double* __restrict__ dphi,
                                                            const double* __restrict__ vol,
                                                            const uint4* __restrict__ telem, int64_t ne,
                                                            unsigned char* __restrict__ blk) {
  using S = typename Pipe32<DIM, DIM>::S;
  const int64_t n = ntiles * kTileElems;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += stride) {
    const int64_t t = w / kTileElems;
    const int k = (int)(w - t * kTileElems);
    const int64_t e = (int64_t)__ldg(ebeg + t) + k;
    const bool in = e < (int64_t)__ldg(ebeg + t + 1);
    unsigned char* B = blk + t * S::kEBytes;
#pragma unroll
    for (int a = 0; a < DIM * DIM; ++a)
      reinterpret_cast<float*>(B + a * S::kArrayBytes)[k] = in ? (float)__ldg(dphi + a * ne + e) : 0.f;
    reinterpret_cast<float*>(B + DIM * DIM * S::kArrayBytes)[k] = in ? (float)__ldg(vol + e) : 0.f;
    reinterpret_cast<uint4*>(B + S::kElemOff)[k] = in ? __ldg(telem + e) : make_uint4(0u, 0u, 0u, 0u);
  }
}

template <int DIM, int D, int MODEL, bool E, bool G, bool DN>
fe_status launch_tile_f32(fe_ctx* c, const ModelParams& mp, double* J, double* dens, double* g, const double* bvp,
                          int nbv) {
  using S = typename Pipe32<DIM, D>::S;
  auto kern = k_tile_f32<DIM, D, MODEL, E, G, DN>;
  static std::atomic<uint64_t> smem_set{0};
  fe_status st = ensure_smem((const void*)kern, c->device, S::kBytes, smem_set);
  if (st) return st;
  TileArgs ta{c->tile_ebeg, c->tile_nbeg, c->tile_node, c->blk32, c->n_tiles, c->n_tpart, c->wait_limit};
  const bool disp = input_is_disp(c);
  const double* b = c->f_host.empty() ? nullptr : c->b;
  const int64_t grid = std::min<int64_t>(c->n_tiles, sm_count(c->device));
  kern<<<(unsigned)grid, kTileThreads, S::kBytes, c->stream>>>(
      ta, c->u_df, b, c->dir, c->eperm, mp, io_perm(c) != nullptr, g, reinterpret_cast<float*>(c->tile_part), dens,
      c->tile_epart, bvp, nbv, disp ? c->bX : 0.0, c->counter, J, c->status);
  return cuda_check(cudaGetLastError(), "f32 tile launch");
}

template <int DIM, int D, int MODEL>
fe_status eval32_t(fe_ctx* c, const double* v, double* J, double* dens, double* g, bool want_energy,
                   bool want_grad) {
  const ModelParams mp = model_params(c);
  const bool E = want_energy, G = want_grad, Dn = dens != nullptr;
  const double* b = c->f_host.empty() ? nullptr : c->b;
  const int nb_node = (int)std::max<int64_t>((c->nn + kThreads - 1) / kThreads, 1);
  double* bvp = c->tile_bvp;
  prof_begin(c, kStagePrep);
  k_pairs32<DIM, D, MODEL><<<nb_node, kThreads, 0, c->stream>>>(c->nn, v, c->X, io_perm(c), E ? b : nullptr, c->u_df,
                                                                 input_is_disp(c), bvp);
  prof_end(c, kStagePrep);
  c->launches++;
  const double* bv_in = (E && b) ? bvp : nullptr;
  prof_begin(c, kStageElem);
  fe_status es;
  if (E && G && Dn) es = launch_tile_f32<DIM, D, MODEL, true, true, true>(c, mp, J, dens, g, bv_in, nb_node);
  else if (E && G) es = launch_tile_f32<DIM, D, MODEL, true, true, false>(c, mp, J, dens, g, bv_in, nb_node);
  else if (E && Dn) es = launch_tile_f32<DIM, D, MODEL, true, false, true>(c, mp, J, dens, g, bv_in, nb_node);
  else if (E) es = launch_tile_f32<DIM, D, MODEL, true, false, false>(c, mp, J, dens, g, bv_in, nb_node);
  else if (G && Dn) es = launch_tile_f32<DIM, D, MODEL, false, true, true>(c, mp, J, dens, g, bv_in, nb_node);
  else if (G) es = launch_tile_f32<DIM, D, MODEL, false, true, false>(c, mp, J, dens, g, bv_in, nb_node);
  else es = launch_tile_f32<DIM, D, MODEL, false, false, true>(c, mp, J, dens, g, bv_in, nb_node);
  prof_end(c, kStageElem);
  if (es) return es;
  c->launches++;
  if (G && c->n_shared > 0) {
    prof_begin(c, kStageGather);
    k_tile_shared<D, PartF32><<<grid_for(c->n_shared * D, kMaxElemBlocks), kThreads, 0, c->stream>>>(
        c->n_shared, c->tile_snode, c->tile_sbeg, c->tile_spart, reinterpret_cast<const float*>(c->tile_part), b,
        c->dir, io_perm(c), g);
    prof_end(c, kStageGather);
    c->launches++;
  }
  return cuda_check(cudaGetLastError(), "eval f32 launch");
}

}  // namespace

size_t tile_block_bytes_f32(int dim) {
  return dim == 3 ? (size_t)Pipe32<3, 3>::S::kEBytes : (size_t)Pipe32<2, 2>::S::kEBytes;
}

fe_status launch_tile_blocks_f32(fe_ctx* c) {
  const int64_t n = c->n_tiles * kTileElems;
  if (n == 0) return FE_OK;
  if (c->dim == 3)
    k_tile_blocks32<3><<<grid_for(n, 4 * kMaxElemBlocks), kThreads, 0, c->stream>>>(
        c->n_tiles, c->tile_ebeg, c->dphi, c->vol, c->tile_elem, c->ne, c->blk32);
  else
    k_tile_blocks32<2><<<grid_for(n, 4 * kMaxElemBlocks), kThreads, 0, c->stream>>>(
        c->n_tiles, c->tile_ebeg, c->dphi, c->vol, c->tile_elem, c->ne, c->blk32);
  c->launches++;
  return cuda_check(cudaGetLastError(), "f32 tile blocks");
}

fe_status launch_eval_f32(fe_ctx* c, const double* v, double* J, double* dens, double* g,
                          bool want_energy, bool want_grad) {
  if (c->model == FE_NEOHOOKE) {
    if (c->dim == 2) return eval32_t<2, 2, FE_NEOHOOKE>(c, v, J, dens, g, want_energy, want_grad);
    return eval32_t<3, 3, FE_NEOHOOKE>(c, v, J, dens, g, want_energy, want_grad);
  }
  if (c->dim == 2) return eval32_t<2, 1, FE_PLAPLACE>(c, v, J, dens, g, want_energy, want_grad);
  return eval32_t<3, 1, FE_PLAPLACE>(c, v, J, dens, g, want_energy, want_grad);
}

}  // namespace fe
