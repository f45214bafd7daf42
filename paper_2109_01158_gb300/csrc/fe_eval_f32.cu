// fe_eval_f32.cu -- the FP32 path (FE_F32_COMP; a precision variant not in the paper): the
// energy J(v) = sum |T| W(F_T) - b.v and its exact gradient (Sec. 5 and 6.2) with the element
// arithmetic in float (elem_f32.cuh) and FP64 energy sums, in one fused persistent launch per
// call plus a small completion launch for the gradient of nodes on tile boundaries.
//
// Persistent blocks (kTileBlocksPerSM per SM) walk their element tiles (fe_tiles.cu,
// tile_common.cuh).  Per tile:
//   B  one thread per element: H from float-pair differences of u, W and |T| dW/dF in float,
//      and the local forces r_{T,l} = |T| dW/dF grad(phi_l) written to the element's local
//      slots in shared memory;
//   C  one thread per tile node: the node's local slots summed in float in a fixed order; a
//      node whose patch lies in the tile gets g_i = sum - b_i (0 on Dirichlet dofs), a shared
//      node leaves its partial sum (slots of one tile are consecutive: coalesced writes);
//   N  the next tile's nodes: u = v - X in FP64 (v in the caller's or the device numbering;
//      u = v for the p-Laplacian or a displacement input), kept as float pairs (hi, lo) so that
//      differences across an element round only once, and the b_i v_i of the nodes this tile
//      owns;
//   the tile's |T| W (summed per thread in float, then per tile in FP64) and b.v go to its
//   energy partial; the last block adds the partials in tile order.
// k_tile_shared adds the shared nodes' partials in tile order.  No intermediate leaves the
// chip except those partials, and every sum has a fixed order (bitwise reproducible, whatever
// the number of blocks).
#include "elem_f32.cuh"
#include "fe_internal.cuh"
#include "tile_common.cuh"

namespace fe {
namespace {

template <int DIM, int D>
struct Pipe32 {
  static constexpr int DP = D == 3 ? 4 : D;   // float pairs per node record (padded)
  static constexpr int NXY = D >= 2 ? 2 : 0;  // components of r kept as float2
  // r: components 0 and 1 as float2 per slot (D >= 2), the last (D = 1 or 3) as float
  using S = TilePipe<DIM, D, 4, DP * 8, D * 4>;
};

template <int D>
__device__ __forceinline__ void load_pairs(const float2* us, int k, float2 (&w)[D]) {
  if constexpr (D == 1) {
    w[0] = us[k];
  } else if constexpr (D == 2) {
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

// N: the float-pair records of a tile's nodes from the copied values V, as (node, component)
// items over the compute threads; returns this thread's b_i v_i over the nodes the tile owns.
template <int DIM, int D, int MODEL>
__device__ __forceinline__ double nodes_to_pairs(const double* V, const int4* rec, int nt, float2* us, bool with_b,
                                                 bool disp, int nthreads) {
  constexpr int DP = Pipe32<DIM, D>::DP;
  double bv = 0.0;
  for (int w = threadIdx.x; w < nt * D; w += nthreads) {
    const int k = w / D, j = w - k * D;
    const double* o = V + k * 3 * D;
    const double vj = o[j];
    us[k * DP + j] = split_double((MODEL == FE_NEOHOOKE && !disp) ? vj - o[D + j] : vj);
    if (with_b && (rec[k].w & 1)) bv = fma(o[2 * D + j], vj, bv);
  }
  return bv;
}

// The block: warps 0 .. kTileElems/32 - 1 compute (one thread per element of a tile, and the
// node work as (node, component) items); the last warp is the producer: its lane 0 issues and
// waits for every bulk copy and loads the tiles' ranges, and the warp adds each tile's energy
// partial.  No compute thread waits on a copy barrier.
template <int DIM, int D, int MODEL, bool ENERGY, bool GRAD, bool DENS>
__global__ void __launch_bounds__(kTileThreads, kTileBlocksPerSM) k_tile_f32(
    TileArgs ta, const double* __restrict__ v, const double* __restrict__ X, const double* __restrict__ b,
    const uint8_t* __restrict__ dir, const int32_t* __restrict__ eperm, ModelParams mp, bool caller_order,
    bool disp, double shift, double* __restrict__ g, float* __restrict__ part, double* __restrict__ dens,
    double* epart, unsigned* counter, double* J, int* status) {
  using P = Pipe32<DIM, D>;
  using S = typename P::S;
  constexpr int K = DIM + 1, NXY = P::NXY, DP = P::DP;
  constexpr int NC = kTileElems;         // compute threads
  constexpr int NCW = NC / 32;           // compute warps
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t barE[2], barR[3];
  __shared__ __align__(16) int4 recs[3][S::kNodes];
  __shared__ int4 info[3];               // {e0, e1, k0, nt} of the tile in each record slot
  __shared__ float ews[NC];               // |T| W of the tile's elements
  __shared__ double wbv[NCW];            // per compute warp: its b.v of the tile
  __shared__ double red[2 * kTileThreads];
  __shared__ int abort_flag;
  float2* us = reinterpret_cast<float2*>(smem + S::kU);
  double* V = reinterpret_cast<double*>(smem + S::kV);
  float2* rxy = reinterpret_cast<float2*>(smem + S::kRs);
  float* rz = reinterpret_cast<float*>(smem + S::kRs + NXY * 4 * S::kSlots);
  const int G = gridDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool compute = tid < NC, producer = warp == NCW, issuer = tid == NC;
  const int64_t ntiles = ta.ntiles;
  const bool with_b = ENERGY && b != nullptr;
  // the issuer's view of the copy pipeline: completed phases and copies in flight per buffer
  uint32_t phE[2] = {0u, 0u}, phR[3] = {0u, 0u, 0u};
  bool pendE[2] = {false, false}, pendR[3] = {false, false, false};
  auto issue_records = [&](int64_t tq, int slot) {
    const int e0 = __ldg(ta.ebeg + tq), e1 = __ldg(ta.ebeg + tq + 1);
    const int k0 = __ldg(ta.nbeg + tq), nt = __ldg(ta.nbeg + tq + 1) - k0;
    info[slot] = make_int4(e0, e1, k0, nt);
    pipe_issue_recs(recs[slot], ta, k0, nt, &barR[slot]);
    pendR[slot] = true;
  };
  auto issue_elems = [&](int slot, int eb) {
    const int4 in = info[slot];
    pipe_issue_elems<S, 4>(smem + S::kE + eb * S::kEBytes, ta, in.x, in.y, &barE[eb]);
    pendE[eb] = true;
  };
  auto wait_e = [&](int eb) {
    const bool ok = mbar_wait_bounded(&barE[eb], phE[eb] & 1u, ta.wait_limit);
    if (ok) { ++phE[eb]; pendE[eb] = false; }
    return ok;
  };
  auto wait_r = [&](int rb) {
    const bool ok = mbar_wait_bounded(&barR[rb], phR[rb] & 1u, ta.wait_limit);
    if (ok) { ++phR[rb]; pendR[rb] = false; }
    return ok;
  };

  int64_t t = blockIdx.x;
  if (issuer) {
    abort_flag = 0;
    for (int q = 0; q < 2; ++q) mbar_init(&barE[q], 1);
    for (int q = 0; q < 3; ++q) mbar_init(&barR[q], 1);
    mbar_init_fence();
    issue_records(t, 0);
    issue_elems(0, 0);
    if (t + G < ntiles) {
      issue_records(t + G, 1);
      issue_elems(1, 1);
    }
    if (!wait_r(0)) abort_flag = 1;
  }
  __syncthreads();
  double bv = 0.0;   // this thread's b_i v_i of the current tile
  if (!abort_flag) {
    if (compute) {
      pipe_gather_nodes<DIM, D, MODEL>(V, recs[0], info[0].w, v, X, with_b ? b : nullptr, caller_order, disp, NC);
      cp_async_wait_all();
    }
    __syncthreads();
    if (compute) bv = nodes_to_pairs<DIM, D, MODEL>(V, recs[0], info[0].w, us, with_b, disp, NC);
    if (issuer) {
      bool ok = wait_e(0);
      if (ok && t + G < ntiles) ok = wait_r(1);
      if (!ok) abort_flag = 1;
    }
  }
  __syncthreads();

  bool bad = false;
  const float C1 = (float)mp.C1, D1 = (float)mp.D1;
  int it = 0;
  for (; t < ntiles && !abort_flag; t += G, ++it) {
    const int eb = it & 1, rb = it % 3, rn = (it + 1) % 3, r2 = (it + 2) % 3;
    const bool has_next = t + G < ntiles, has_t2 = t + 2 * (int64_t)G < ntiles;
    const int4 in = info[rb];
    const int e0 = in.x, e1 = in.y, nt = in.w;
    const int ntn = has_next ? info[rn].w : 0;
    const int4* R = recs[rb];
    const unsigned char* E = smem + S::kE + eb * S::kEBytes;

    if (producer) {
      // the records of the tile after next (slot r2 held the previous tile's)
      if (issuer && has_t2) issue_records(t + 2 * (int64_t)G, r2);
    } else {
      // the next tile's nodal values start copying
      if (has_next)
        pipe_gather_nodes<DIM, D, MODEL>(V, recs[rn], ntn, v, X, with_b ? b : nullptr, caller_order, disp, NC);

      // B: one thread per element
      float ew = 0.f;   // this thread's |T| W
      const int e = e0 + tid;
      if (e < e1) {
        const int el = tid;
        const uint4 le = reinterpret_cast<const uint4*>(E + S::kElemOff)[el];
        const int lid[4] = {(int)(le.x & 0xffffu), (int)(le.x >> 16), (int)(le.y & 0xffffu), (int)(le.y >> 16)};
        float2 u0[D], ul[D];
        load_pairs<D>(us, lid[0], u0);
        float a[DIM][D];
#pragma unroll
        for (int l = 1; l < K; ++l) {
          load_pairs<D>(us, lid[l], ul);
#pragma unroll
          for (int j = 0; j < D; ++j) a[l - 1][j] = pair_diff(ul[j], u0[j]);
        }
        float gg[DIM][DIM];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
          for (int m = 0; m < DIM; ++m) gg[l][m] = reinterpret_cast<const float*>(E + (l * DIM + m) * S::kArrayBytes)[el];
        const float vT = reinterpret_cast<const float*>(E + DIM * DIM * S::kArrayBytes)[el];
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
            if constexpr (NXY) rxy[sl[l]] = make_float2(r[0], r[1]);
            if constexpr (D != 2) rz[sl[l]] = r[D - 1];
          }
          if constexpr (NXY) rxy[sl[0]] = make_float2(r0[0], r0[1]);
          if constexpr (D != 2) rz[sl[0]] = r0[D - 1];
        }
      }
      if (ENERGY) {
        ews[tid] = ew;
        if (with_b) {
          const double wb = pipe_warp_sum(bv);
          if (lane == 0) wbv[warp] = wb;
        }
      }
    }
    __syncthreads();

    if (producer) {
      // the element stage of this tile is free: the element copies of the tile after next
      if (issuer && has_t2) issue_elems(r2, eb);
      // the tile's energy partial, in FP64 from the compute warps' float pairs
      if (ENERGY) {
        const double x = pipe_warp_sum_floats(ews, NC);
        double xb = 0.0;
        if (with_b) xb = pipe_warp_sum(lane < NCW ? wbv[lane] : 0.0);
        if (lane == 0) {
          epart[t] = x;
          epart[ntiles + t] = xb;
        }
      }
    } else {
      // C: patch sums, one thread per tile node
      if (GRAD) {
        for (int k = tid; k < nt; k += NC) {
          const int4 rec = R[k];
          const int beg = rec.z & 0xffff, cnt = (int)((unsigned)rec.z >> 16);
          // walk the node's slots from position k mod cnt, wrapping around: consecutive nodes
          // then start on different shared-memory banks; the order is fixed by the mesh alone
          float s[D];
#pragma unroll
          for (int j = 0; j < D; ++j) s[j] = 0.f;
          if (cnt > 0) {
            const int p = (int)((unsigned)k % (unsigned)cnt);
            auto add = [&](int q, bool first) {
              if constexpr (NXY) {
                const float2 xy = rxy[q];
                s[0] = first ? xy.x : __fadd_rn(s[0], xy.x);
                s[1] = first ? xy.y : __fadd_rn(s[1], xy.y);
              }
              if constexpr (D != 2) s[D - 1] = first ? rz[q] : __fadd_rn(s[D - 1], rz[q]);
            };
            add(beg + p, true);
#pragma unroll 4
            for (int q = beg + p + 1; q < beg + cnt; ++q) add(q, false);
#pragma unroll 4
            for (int q = beg; q < beg + p; ++q) add(q, false);
          }
          const int dst = (rec.w >> 1) - 1;
          const int64_t i = rec.x;
          if (dst < 0) {
            const int64_t o = caller_order ? (int64_t)rec.y : i;
#pragma unroll
            for (int j = 0; j < D; ++j) {
              const double sj = f2d_bits(s[j]);
              g[o * D + j] = __ldg(dir + i * D + j) ? 0.0 : (b ? sj - __ldg(b + i * D + j) : sj);
            }
          } else {
#pragma unroll
            for (int j = 0; j < D; ++j) part[(int64_t)dst * D + j] = s[j];
          }
        }
      }
      cp_async_wait_all();
    }
    __syncthreads();

    // N: the next tile's nodes; the issuer waits for the next tile's elements and for the
    // records of the tile after next
    if (has_next) {
      if (issuer) {
        bool ok = wait_e(eb ^ 1);
        if (ok && has_t2) ok = wait_r(r2);
        if (!ok) abort_flag = 1;
      }
      if (compute) bv = nodes_to_pairs<DIM, D, MODEL>(V, recs[rn], ntn, us, with_b, disp, NC);
    }
    __syncthreads();
  }

  if (abort_flag) {
    // a copy did not arrive in time: record it, wait with the full limit for every copy still
    // in flight (nothing may land in shared memory after the block has left), and make J NaN
    cp_async_wait_all();
    if (issuer) {
      atomicOr(status, kStatusTimeout);
      for (int q = 0; q < 2; ++q)
        if (pendE[q]) mbar_wait_bounded(&barE[q], phE[q] & 1u);
      for (int q = 0; q < 3; ++q)
        if (pendR[q]) mbar_wait_bounded(&barR[q], phR[q] & 1u);
    }
    if (ENERGY && producer && lane == 0)
      for (int64_t tq = t; tq < ntiles; tq += G) {
        epart[tq] = CUDART_NAN;
        epart[ntiles + tq] = 0.0;
      }
  }
  if (ENERGY && producer && lane == 0) __threadfence();   // this block's partials, before the ticket
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) pipe_finish_energy(epart, ntiles, shift, counter, J, red);
}

template <int DIM, int D, int MODEL, bool E, bool G, bool DN>
fe_status launch_tile_f32(fe_ctx* c, const ModelParams& mp, const double* v, double* J, double* dens, double* g) {
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
  const int64_t grid = std::min<int64_t>(c->n_tiles, (int64_t)kTileBlocksPerSM * sm_count(c->device));
  kern<<<(unsigned)grid, kTileThreads, S::kBytes, c->stream>>>(
      ta, v, c->X, b, c->dir, c->eperm, mp, io_perm(c) != nullptr, disp, disp ? c->bX : 0.0, g,
      reinterpret_cast<float*>(c->tile_part), dens, c->tile_epart, c->counter, J, c->status);
  return cuda_check(cudaGetLastError(), "f32 tile launch");
}

template <int DIM, int D, int MODEL>
fe_status eval32_t(fe_ctx* c, const double* v, double* J, double* dens, double* g, bool want_energy,
                   bool want_grad) {
  const ModelParams mp = model_params(c);
  const bool E = want_energy, G = want_grad, Dn = dens != nullptr;
  prof_begin(c, kStageElem);
  fe_status es;
  if (E && G && Dn) es = launch_tile_f32<DIM, D, MODEL, true, true, true>(c, mp, v, J, dens, g);
  else if (E && G) es = launch_tile_f32<DIM, D, MODEL, true, true, false>(c, mp, v, J, dens, g);
  else if (E && Dn) es = launch_tile_f32<DIM, D, MODEL, true, false, true>(c, mp, v, J, dens, g);
  else if (E) es = launch_tile_f32<DIM, D, MODEL, true, false, false>(c, mp, v, J, dens, g);
  else if (G && Dn) es = launch_tile_f32<DIM, D, MODEL, false, true, true>(c, mp, v, J, dens, g);
  else if (G) es = launch_tile_f32<DIM, D, MODEL, false, true, false>(c, mp, v, J, dens, g);
  else es = launch_tile_f32<DIM, D, MODEL, false, false, true>(c, mp, v, J, dens, g);
  prof_end(c, kStageElem);
  if (es) return es;
  c->launches++;
  if (G && c->n_shared > 0) {
    prof_begin(c, kStageGather);
    const double* b = c->f_host.empty() ? nullptr : c->b;
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
