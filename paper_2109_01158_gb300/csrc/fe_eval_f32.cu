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
//                   node warps copy the next tile's float pairs into shared memory;
//                   element warps, one thread per element: H from float-pair differences of
//                      u, W and |T| dW/dF in float, and the local forces
//                      r_{T,l} = |T| dW/dF grad(phi_l) written to the element's local slots in
//                      shared memory;
//                   node warps then sum the patches, one thread per tile node: the node's
//                      local slots summed in float in a fixed order; a node whose patch lies
//                      in the tile gets g_i = sum - b_i (0 on Dirichlet dofs), a shared node
//                      leaves its partial sum;
//                   the producer warp issues the bulk copies and adds the tile's |T| W into its
//                      energy partial (float pairs per lane, FP64 across lanes); the last block
//                      adds the partials in tile order;
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
    const int64_t src = perm ? (int64_t)__ldg(perm + i) : i;
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
  uint64_t e_full[2], e_empty[2];    // element stage: TMA landed / element warps done
  uint64_t r_full[3], r_empty[3];    // node records: TMA landed / node warps done
  uint64_t u_full[2], u_empty[2];    // nodal values: node warps wrote / element warps done
  uint64_t rs_full[2], rs_empty[2];  // local forces and energies: element warps wrote / node
                                     // warps and producer done
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
  __shared__ int4 info[3];        // {e0, e1, k0, nt} of the tile whose records are in R[slot]
  __shared__ volatile int abort_flag;
  const int G = gridDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool elem_warp = warp < NEW, node_warp = !elem_warp && warp < NEW + kTileNodeWarps;
  const bool issuer = tid == NE + NN;
  const int64_t ntiles = ta.ntiles;
  const int my_tiles = (int)((ntiles - blockIdx.x + G - 1) / G);   // tiles blockIdx.x + i G
  auto tile_of = [&](int i) { return (int64_t)blockIdx.x + (int64_t)i * G; };
  auto E = [&](int i) { return smem + S::kE + (i & 1) * S::kEBytes; };
  auto R = [&](int i) { return reinterpret_cast<int4*>(smem + S::kR + (i % 3) * S::kRBytes); };
  auto U = [&](int i) { return reinterpret_cast<float2*>(smem + S::kU + (i & 1) * S::kUBytes); };
  // component j of the local forces of tile i, by local slot
  auto RC = [&](int i, int j) { return reinterpret_cast<float*>(smem + S::kRs + (i & 1) * S::kRsBytes + j * S::kColBytes); };
  auto EW = [&](int i) { return reinterpret_cast<float*>(smem + S::kEw + (i & 1) * S::kEwBytes); };
  auto BDB = [&](int i) { return reinterpret_cast<double*>(smem + S::kBd + (i % 3) * S::kBdBytes); };
  auto BDM = [&](int i) { return reinterpret_cast<int*>(smem + S::kBd + (i % 3) * S::kBdBytes + S::kBdMaskOff); };
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
  int nE[2] = {0, 0}, nR[3] = {0, 0, 0};
  auto issue_elems = [&](int i) {
    const int4 in = info[i % 3];
    pipe_issue_elems<S, 4>(E(i), ta, in.x, in.y, &bars.e_full[i & 1]);
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
    info[i % 3] = make_int4(raw.x, raw.y, raw.z, raw.w - raw.z);
    pipe_issue_recs(R(i), ta, raw.z, raw.w - raw.z, &bars.r_full[i % 3]);
    ++nR[i % 3];
    load_pre(i + 1);
  };
  if (tid == 0) abort_flag = 0;
  if (issuer) {
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bars.e_full[q], 1);
      mbar_init(&bars.e_empty[q], NEW);
      mbar_init(&bars.u_full[q], kTileNodeWarps);
      mbar_init(&bars.u_empty[q], NEW);
      mbar_init(&bars.rs_full[q], NEW);
      mbar_init(&bars.rs_empty[q], NEW + 1);
    }
    for (int q = 0; q < 3; ++q) {
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
      // records of the first three tiles, elements of the first two
      for (int i = 0; i < 3 && i < my_tiles; ++i) issue_recs(i);
      for (int i = 0; i < 2 && i < my_tiles; ++i) issue_elems(i);
    }
    for (int i = 0; i < my_tiles; ++i) {
      // the element stage of tile i is free once the element warps are done with it (the same
      // moment as their forces and energies are complete)
      if (i + 2 < my_tiles) {
        if (!wait_lane0(&bars.e_empty[i & 1], i >> 1)) break;
        if (issuer) issue_elems(i + 2);
      }
      if (!wait(&bars.rs_full[i & 1], i >> 1)) break;
      if (ENERGY) {
        // the element warps' pairs, in FP64 across lanes in a fixed order
        const float2 wp = lane < NEW ? reinterpret_cast<const float2*>(EW(i))[lane] : make_float2(0.f, 0.f);
        const bool inf = __any_sync(0xffffffffu, isinf(wp.x));
        double x = pipe_warp_sum(f2d_bits(wp.x) + f2d_bits(wp.y));
        if (inf) x = CUDART_INF;
        if (lane == 0) epart[tile_of(i)] = x;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.rs_empty[i & 1]);
      // the record slot of tile i is free once the node warps have summed its patches
      if (i + 3 < my_tiles) {
        if (!wait_lane0(&bars.r_empty[i % 3], i / 3)) break;
        if (issuer) issue_recs(i + 3);
      }
    }
  } else if (node_warp) {
    const int ntid = tid - NE;
    // the nodal values of tile i (its records must have landed) into U(i)
    auto gather = [&](int i) {
      if (!wait(&bars.r_full[i % 3], i / 3)) return false;
      if (i >= 2 && !wait(&bars.u_empty[i & 1], (i >> 1) - 1)) return false;
      const int4* rec = R(i);
      float2* us = U(i);
      const int nt = info[i % 3].w;
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
          const int64_t n = rec[k].x;
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
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.u_full[i & 1]);
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
        const int nt = info[i % 3].w;
        for (int w = tid; w < nt * D; w += NE) {
          const int k = w / D, j = w - k * D;
          const int4 rec = Rr[k];
          const int beg = rec.z & 0xffff, cnt = (int)((unsigned)rec.z >> 16);
          // the node's slots in order (each node's slots are consecutive in its column)
          const float* col = rc0 + j * (S::kColBytes / 4) + beg;
          float sum = 0.f;
          if (cnt > 0) {
            sum = col[0];
#pragma unroll 4
            for (int q = 1; q < cnt; ++q) sum = __fadd_rn(sum, col[q]);
          }
          const int dst = (rec.w >> 1) - 1;
          const int64_t n = rec.x;
          if (dst < 0) {
            const int64_t o = caller_order ? (int64_t)rec.y : n;
            g[o * D + j] = ((bm[k] >> j) & 1) ? 0.0 : f2d_bits(sum) - bd[k * D + j];
          } else {
            part[(int64_t)dst * D + j] = sum;
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars.rs_empty[i & 1]);
        mbar_arrive(&bars.r_empty[i % 3]);
      }
      return true;
    };
    for (int i = 0; i < my_tiles && ok; ++i) {
      // B: one thread per element of tile i
      if (!wait(&bars.e_full[i & 1], i >> 1) || !wait(&bars.u_full[i & 1], i >> 1)) break;
      if (i >= 2 && !wait(&bars.rs_empty[i & 1], (i >> 1) - 1)) break;
      const int4 in = info[i % 3];
      const unsigned char* St = E(i);
      const float2* us = U(i);
      float* rc0 = RC(i, 0);
      float ew = 0.f;
      const int e = in.x + tid;
      if (e < in.y) {
        const uint4 le = reinterpret_cast<const uint4*>(St + S::kElemOff)[tid];
        const int lid[4] = {(int)(le.x & 0xffffu), (int)(le.x >> 16), (int)(le.y & 0xffffu), (int)(le.y >> 16)};
        float a[DIM][D];
#pragma unroll
        for (int l = 1; l < K; ++l)
#pragma unroll
          for (int j = 0; j < D; ++j) a[l - 1][j] = pair_diff(us[lid[l] * DP + j], us[lid[0] * DP + j]);
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
          const int sl[4] = {(int)(le.z & 0xffffu), (int)(le.z >> 16), (int)(le.w & 0xffffu), (int)(le.w >> 16)};
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
        // the warp's |T| W as a float pair: a fixed TwoSum tree over the lanes (+Inf apart,
        // as TwoSum on Inf gives NaN); the producer adds the tile's warp pairs in FP64
        const bool inf = __any_sync(0xffffffffu, isinf(ew));
        df p = {isinf(ew) ? 0.f : ew, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const df q = {__shfl_down_sync(0xffffffffu, p.hi, o), __shfl_down_sync(0xffffffffu, p.lo, o)};
          p = df_add(p, q);
        }
        if (lane == 0) reinterpret_cast<float2*>(EW(i))[warp] = inf ? make_float2(CUDART_INF_F, 0.f) : make_float2(p.hi, p.lo);
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars.e_empty[i & 1]);
        mbar_arrive(&bars.u_empty[i & 1]);
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
      for (int q = 0; q < 3; ++q)
        if (nR[q] > 0) mbar_wait_bounded(&bars.r_full[q], (uint32_t)(nR[q] - 1) & 1u);
      if (ENERGY)
        for (int i = 0; i < my_tiles; ++i) epart[tile_of(i)] = CUDART_NAN;
    }
  }
  if (ENERGY && warp == NEW + kTileNodeWarps && lane == 0) __threadfence();   // partials before the ticket
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) pipe_finish_energy(epart, ntiles, bvp, nbv, shift, counter, J, reinterpret_cast<double*>(smem + S::kRs));
}

template <int DIM, int D, int MODEL, bool E, bool G, bool DN>
fe_status launch_tile_f32(fe_ctx* c, const ModelParams& mp, double* J, double* dens, double* g, const double* bvp,
                          int nbv) {
  using S = typename Pipe32<DIM, D>::S;
  auto kern = k_tile_f32<DIM, D, MODEL, E, G, DN>;
  static std::atomic<uint64_t> smem_set{0};
  fe_status st = ensure_smem((const void*)kern, c->device, S::kBytes, smem_set);
  if (st) return st;
  TileArgs ta{c->tile_ebeg, c->tile_nbeg, c->tile_node, reinterpret_cast<const unsigned char*>(c->dphi32),
              reinterpret_cast<const unsigned char*>(c->vol32), c->tile_elem, c->n_tiles, padded_ne(c->ne),
              c->wait_limit};
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
