// fe_eval_f32.cu -- FP32 element arithmetic with compensated reductions (not in the paper).
//
// The element work of Sec. 5 / 6.2 in float, written in displacement form so that no
// O(1) quantities cancel: with F = I + H (H = grad u, u = v - X),
//   delta = det F - 1 = tr H + i2(H) + det H      (i2: sum of principal 2x2 minors; 2D: tr H + det H)
//   I1 - dim - 2 log det F = |H|^2 - 2 (i2(H) + det H) + 2 phi(delta),   phi(x) = x - log(1+x)
//   dW/dF = 2 C1 (F - F^{-T}) + 2 D1 delta cof F,   F - F^{-T} = H + cof(F) H^T / det F
// phi uses the series of 2 atanh: with s = x/(2+x), log(1+x) = 2(s + s^3/3 + s^5/5 + ...),
// so phi(x) = s x - 2 s^3 (1/3 + s^2/5 + s^4/7 + ...).  Where |delta| > 1/2, or det F is
// close to 0, delta and log det F are taken in FP64.
//
// Reductions: each thread accumulates |T| W in a float pair (TwoSum, Knuth), the pair is
// converted to double per thread, and the block/global trees run in double.  The patch
// sums of the gradient are float pairs converted to double per node.  No floating-point
// operation is done in FP64 per element except in the rare FP64 branch above.
#include "fe_internal.cuh"
#include "gather_bulk.cuh"
#include "tile_stream.cuh"

namespace fe {
namespace {

// ---- float-pair accumulation (error-free TwoSum) ---------------------------------------
struct FPair {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const df t = two_sum(hi, x);
    hi = t.hi;
    lo = fadd(lo, t.lo);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double block_sum(double x, double* sh) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  x = (threadIdx.x < kThreads / 32) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) x = warp_sum(x);
  __syncthreads();
  return x;
}

__device__ __forceinline__ void finish_energy(double block_total, double* partials, int n_elem_blocks,
                                              const double* node_partials, int n_node_blocks,
                                              unsigned* counter, double* J, double* sh) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = block_total;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == (unsigned)n_elem_blocks - 1u);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double s = 0.0, t = 0.0;
  for (int k = threadIdx.x; k < n_elem_blocks; k += kThreads) s += __ldcg(partials + k);
  for (int k = threadIdx.x; k < n_node_blocks; k += kThreads) t += __ldcg(node_partials + k);
  s = block_sum(s, sh);
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    *J = s - t;
    *counter = 0u;
  }
}

// phi(x) = x - log(1+x) for |x| <= 1/2 by the atanh series (|s| <= 1/3, 8 terms).
__device__ __forceinline__ float phi_series(float x) {
  const float s = x / (2.0f + x);
  const float s2 = s * s;
  float t = 1.0f / 17.0f;
  t = fmaf(t, s2, 1.0f / 15.0f);
  t = fmaf(t, s2, 1.0f / 13.0f);
  t = fmaf(t, s2, 1.0f / 11.0f);
  t = fmaf(t, s2, 1.0f / 9.0f);
  t = fmaf(t, s2, 1.0f / 7.0f);
  t = fmaf(t, s2, 1.0f / 5.0f);
  t = fmaf(t, s2, 1.0f / 3.0f);
  return fmaf(s, x, -2.0f * s * s2 * t);
}

// det F, 2 (delta - log det F) and 1 / det F in FP64 from the float entries of H (F = I + H);
// returns false if det F <= 0.
__device__ __noinline__ bool far_from_identity_f64(const float* Hf, int dim, float* delta, float* phi2,
                                                   float* inv_det) {
  double detd;
  if (dim == 3) {
    const double F00 = 1.0 + Hf[0], F11 = 1.0 + Hf[4], F22 = 1.0 + Hf[8];
    const double H01 = Hf[1], H02 = Hf[2], H10 = Hf[3], H12 = Hf[5], H20 = Hf[6], H21 = Hf[7];
    detd = F00 * (F11 * F22 - H12 * H21) + H01 * (H12 * H20 - H10 * F22) + H02 * (H10 * H21 - F11 * H20);
  } else {
    detd = (1.0 + Hf[0]) * (1.0 + Hf[3]) - (double)Hf[1] * (double)Hf[2];
  }
  if (!(detd > 0.0)) {
    *delta = 0.f;
    *phi2 = 0.f;
    *inv_det = 1.f;
    return false;
  }
  const double dd = detd - 1.0;
  *delta = (float)dd;
  *phi2 = (float)(2.0 * (dd - log(detd)));
  *inv_det = (float)(1.0 / detd);
  return true;
}

// Node record of the displacement as double-float pairs (D pairs, padded to 4 in 3D).  The
// float path rounds only the differences u_l - u_0 to float: the displacement itself can be
// hundreds of times larger than its differences across an element, and rounding it first
// would lose that factor in grad u.
template <int D>
__device__ __forceinline__ void load_u_pairs(const float2* __restrict__ u, int32_t n, df* out) {
  if (D == 1) {
    const float2 a = __ldg(u + n);
    out[0] = {a.x, a.y};
  } else if (D == 2) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(u) + n);
    out[0] = {a.x, a.y};
    out[1] = {a.z, a.w};
  } else {
    const float4* p = reinterpret_cast<const float4*>(u) + 2 * (int64_t)n;
    const float4 a = __ldg(p), b = __ldg(p + 1);
    out[0] = {a.x, a.y};
    out[1] = {a.z, a.w};
    out[2] = {b.x, b.y};
  }
}

template <int D, bool NH, int DIM>
__global__ void __launch_bounds__(kThreads) k_node_prep32(int64_t nn, const double* __restrict__ v,
                                                          const double* __restrict__ X,
                                                          const int32_t* __restrict__ perm,
                                                          const double* __restrict__ b,
                                                          float2* __restrict__ u,
                                                          double* __restrict__ node_partials, bool disp,
    double shift) {
  __shared__ double sh[kThreads / 32];
  constexpr int DP = D == 3 ? 4 : D;
  double dot = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    const int64_t src = perm ? (int64_t)perm[i] : i;
    df w[DP];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const double vj = v[src * D + j];
      dot += b[i * D + j] * vj;
      w[j] = df_from_double((NH && !disp) ? vj - X[i * DIM + j] : vj);
    }
    if (DP == 4) w[3] = {0.f, 0.f};
    if (DP == 1) {
      u[i] = make_float2(w[0].hi, w[0].lo);
    } else {
      float4* o = reinterpret_cast<float4*>(u) + i * (DP / 2);
      o[0] = make_float4(w[0].hi, w[0].lo, w[1].hi, w[1].lo);
      if (DP == 4) o[1] = make_float4(w[2].hi, w[2].lo, w[3].hi, w[3].lo);
    }
  }
  dot = block_sum(dot, sh);
  // block 0 adds b.X when v is a displacement (then dot sums b.u)
  if (threadIdx.x == 0) node_partials[blockIdx.x] = (blockIdx.x == 0 && disp) ? dot + shift : dot;
}

template <int DIM, bool GRAD>
struct F32Arrays {
  static constexpr int K = DIM + 1;
  static constexpr int kDphi = 0;                  // DIM*DIM arrays of float
  static constexpr int kVol = DIM * DIM;           // float
  static constexpr int kElems = DIM * DIM + 1;     // K arrays of int32
  static constexpr int kSlots = kElems + K;        // K arrays of int32 (gradient only)
  static constexpr int N = kSlots + (GRAD ? K : 0);
};

template <int NT>
__device__ __forceinline__ double block_sum_nt(double x, double* sh) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  x = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
  if (warp == 0) x = warp_sum(x);
  __syncthreads();
  return x;
}

template <int NT>
__device__ __forceinline__ void finish_energy_nt(double block_total, double* partials, int n_elem_blocks,
                                                 const double* node_partials, int n_node_blocks,
                                                 unsigned* counter, double* J, double* sh) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = block_total;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == (unsigned)n_elem_blocks - 1u);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double s = 0.0, t = 0.0;
  for (int k = threadIdx.x; k < n_elem_blocks; k += NT) s += __ldcg(partials + k);
  for (int k = threadIdx.x; k < n_node_blocks; k += NT) t += __ldcg(node_partials + k);
  s = block_sum_nt<NT>(s, sh);
  t = block_sum_nt<NT>(t, sh);
  if (threadIdx.x == 0) {
    *J = s - t;
    *counter = 0u;
  }
}

// Element kernel: persistent blocks stream tiles of the element arrays through shared-memory
// stages with bulk copies (tile_stream.cuh); one element per thread and tile.
template <int DIM, int D, int MODEL, bool ENERGY, bool GRAD, bool DENS>
__global__ void __launch_bounds__(kTile, kTileMinBlocks) k_elem_f32(
    int64_t ne, TileArrays<F32Arrays<DIM, GRAD>::N> A, const float2* __restrict__ u,
    const int32_t* __restrict__ eperm, ModelParams mp, float* __restrict__ r,
    double* __restrict__ dens, double* partials, const double* node_partials, int n_node_blocks,
    unsigned* counter, double* J, int* status) {
  constexpr int K = DIM + 1;
  using AR = F32Arrays<DIM, GRAD>;
  constexpr int NA = AR::N;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ double sh[kTile / 32];
  TileLayout<NA> L;
  L.init(A);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < kStages; ++k) mbar_init(&bars[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int64_t ntiles = (ne + kTile - 1) / kTile;
  if (threadIdx.x == 0)
    for (int k = 0; k < kStages; ++k) {
      const int64_t t = blockIdx.x + (int64_t)k * gridDim.x;
      if (t < ntiles) tile_issue(A, L, smem + k * L.stage_bytes, &bars[k], t, ne);
    }
  FPair acc;
  bool bad = false, inf_seen = false;
  const float C1 = (float)mp.C1, D1 = (float)mp.D1;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int sidx = it % kStages;
    unsigned char* st = smem + sidx * L.stage_bytes;
    const bool ok = mbar_wait_bounded(&bars[sidx], (uint32_t)((it / kStages) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(status, kStatusTimeout);
        for (int k = 0; k < kStages; ++k) {
          const int64_t t = tile + (int64_t)k * gridDim.x;
          if (t < ntiles) mbar_wait_bounded(&bars[(it + k) % kStages], (uint32_t)(((it + k) / kStages) & 1));
        }
      }
      return;
    }
    const int tid = threadIdx.x;
    const int64_t e = tile * kTile + tid;
    if (e < ne) {
    df ul[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) load_u_pairs<D>(u, tile_get<int32_t>(st, L, AR::kElems + l, tid, 4), ul[l]);
    float g[DIM][DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = tile_get<float>(st, L, AR::kDphi + l * DIM + m, tid, 4);
    const float vT = tile_get<float>(st, L, AR::kVol, tid, 4);
    float H[D][DIM];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      // u_l - u_0 to float accuracy from the pairs: the hi difference is exact when the two
      // values are within a factor 2 (Sterbenz' lemma), otherwise within half an ulp of a
      // result of the same size; adding the (tiny) lo difference and rounding once leaves at
      // most about one float ulp of the difference
      float a[DIM];
#pragma unroll
      for (int l = 0; l < DIM; ++l)
        a[l] = fadd(fsub(ul[l + 1][j].hi, ul[0][j].hi), fsub(ul[l + 1][j].lo, ul[0][j].lo));
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        float s = a[0] * g[0][m];
#pragma unroll
        for (int l = 1; l < DIM; ++l) s = fmaf(a[l], g[l][m], s);
        H[j][m] = s;
      }
    }
    float W = 0.f;
    float P[D][DIM];
    if (MODEL == FE_NEOHOOKE) {
      float hsq = 0.f;
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) hsq = fmaf(H[j][m], H[j][m], hsq);
      float tr, i2, dH, C[DIM][DIM];  // C = cof(I + H)
      if (DIM == 3) {
        tr = H[0][0] + H[1][1] + H[2][2];
        i2 = (H[0][0] * H[1][1] - H[0][1] * H[1][0]) + (H[0][0] * H[2][2] - H[0][2] * H[2][0]) +
             (H[1][1] * H[2][2] - H[1][2] * H[2][1]);
        const float m00 = H[1][1] * H[2][2] - H[1][2] * H[2][1];
        const float m01 = H[1][2] * H[2][0] - H[1][0] * H[2][2];
        const float m02 = H[1][0] * H[2][1] - H[1][1] * H[2][0];
        dH = H[0][0] * m00 + H[0][1] * m01 + H[0][2] * m02;
        if (GRAD) {
          const float F00 = 1.f + H[0][0], F11 = 1.f + H[1][1], F22 = 1.f + H[2][2];
          C[0][0] = F11 * F22 - H[1][2] * H[2][1];
          C[0][1] = H[1][2] * H[2][0] - H[1][0] * F22;
          C[0][2] = H[1][0] * H[2][1] - F11 * H[2][0];
          C[1][0] = H[0][2] * H[2][1] - H[0][1] * F22;
          C[1][1] = F00 * F22 - H[0][2] * H[2][0];
          C[1][2] = H[0][1] * H[2][0] - F00 * H[2][1];
          C[2][0] = H[0][1] * H[1][2] - H[0][2] * F11;
          C[2][1] = H[0][2] * H[1][0] - F00 * H[1][2];
          C[2][2] = F00 * F11 - H[0][1] * H[1][0];
        }
      } else {
        tr = H[0][0] + H[1][1];
        dH = H[0][0] * H[1][1] - H[0][1] * H[1][0];
        i2 = 0.f;
        if (GRAD) {
          C[0][0] = 1.f + H[1][1];
          C[0][1] = -H[1][0];
          C[1][0] = -H[0][1];
          C[1][1] = 1.f + H[0][0];
        }
      }
      float delta = tr + i2 + dH;
      bool ebad = false;
      float phi2;      // 2 phi(delta)
      float inv_det;   // 1 / det F
      const bool far = !(fabsf(delta) <= 0.5f);
      if (!far) {
        phi2 = 2.f * phi_series(delta);
        inv_det = 1.f / (1.f + delta);
      }
      // Far from F = I: det F and log det F in FP64, in a called function behind a warp
      // vote so that the compiler cannot if-convert it into every element's path.
      if (__any_sync(__activemask(), far) && far) {
        float Hf[9];
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
          for (int m = 0; m < DIM; ++m) Hf[j * DIM + m] = H[j][m];
        ebad = !far_from_identity_f64(Hf, DIM, &delta, &phi2, &inv_det);
      }
      if (ENERGY || DENS) W = C1 * (hsq - 2.f * (i2 + dH) + phi2) + D1 * delta * delta;
      if (ebad) {
        W = CUDART_INF_F;
        bad = true;
      }
      if (GRAD) {
        // P = 2 C1 (H + C H^T / det F) + 2 D1 delta C, scaled by |T|
        const float a = 2.f * C1 * vT, c = 2.f * D1 * delta * vT, ai = a * inv_det;
#pragma unroll
        for (int j = 0; j < DIM; ++j)
#pragma unroll
          for (int m = 0; m < DIM; ++m) {
            float ch = 0.f;  // (C H^T)_jm = sum_k C_jk H_mk
#pragma unroll
            for (int k = 0; k < DIM; ++k) ch = fmaf(C[j][k], H[m][k], ch);
            P[j][m] = fmaf(a, H[j][m], fmaf(ai, ch, c * C[j][m]));
          }
      }
    } else {
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < DIM; ++m) s = fmaf(H[0][m], H[0][m], s);
      if (ENERGY || DENS) {
        if (mp.pcase == 2) W = 0.5f * s;
        else if (mp.pcase == 3) W = s * sqrtf(s) * (1.f / 3.f);
        else W = s > 0.f ? powf(s, 0.5f * (float)mp.p) / (float)mp.p : 0.f;
      }
      if (GRAD) {
        float cf = (mp.pcase == 2) ? 1.f : (mp.pcase == 3) ? sqrtf(s)
                                     : (s > 0.f ? powf(s, 0.5f * (float)(mp.p - 2.0)) : 0.f);
        cf *= vT;
#pragma unroll
        for (int m = 0; m < DIM; ++m) P[0][m] = cf * H[0][m];
      }
    }
    if (ENERGY) {
      if (isinf(W)) inf_seen = true;   // +Inf would become NaN inside TwoSum
      else acc.add(vT * W);
    }
    if (DENS) dens[eperm ? (int64_t)eperm[e] : e] = (double)W;
    if (GRAD) {
      float r0[D];
#pragma unroll
      for (int l = 1; l <= DIM; ++l) {
        const int64_t q = tile_get<int32_t>(st, L, AR::kSlots + l, tid, 4);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          float s = P[j][0] * g[l - 1][0];
#pragma unroll
          for (int m = 1; m < DIM; ++m) s = fmaf(P[j][m], g[l - 1][m], s);
          r[q * D + j] = s;
          r0[j] = (l == 1) ? -s : r0[j] - s;
        }
      }
      const int64_t q0 = tile_get<int32_t>(st, L, AR::kSlots, tid, 4);
#pragma unroll
      for (int j = 0; j < D; ++j) r[q0 * D + j] = r0[j];
    }
    }
    __syncthreads();   // every thread is done with this stage
    const int64_t nxt = tile + (int64_t)kStages * gridDim.x;
    if (threadIdx.x == 0 && nxt < ntiles) tile_issue(A, L, st, &bars[sidx], nxt, ne);
  }
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) {
    const double t = block_sum_nt<kTile>(inf_seen ? CUDART_INF : acc.value(), sh);
    finish_energy_nt<kTile>(t, partials, gridDim.x, node_partials, n_node_blocks, counter, J, sh);
  }
}

template <int DIM, int D, int MODEL, bool E, bool G, bool DN>
fe_status launch_elem_f32(fe_ctx* c, const ModelParams& mp, double* dens, const double* node_partials,
                          int nb_node, double* J) {
  using AR = F32Arrays<DIM, G>;
  TileArrays<AR::N> A;
  int stage_bytes = 0;
  for (int a = 0; a < AR::N; ++a) {
    const unsigned char* base;
    if (a < AR::kVol) base = reinterpret_cast<const unsigned char*>(c->dphi32 + (int64_t)a * c->ne);
    else if (a == AR::kVol) base = reinterpret_cast<const unsigned char*>(c->vol32);
    else if (a < AR::kSlots) base = reinterpret_cast<const unsigned char*>(c->elems + (int64_t)(a - AR::kElems) * c->ne);
    else base = reinterpret_cast<const unsigned char*>(c->slot + (int64_t)(a - AR::kSlots) * c->ne);
    A.base[a] = base;
    A.esize[a] = 4;
    stage_bytes += ((kTile * 4 + 16) + 15) & ~15;
  }
  const int smem = kStages * stage_bytes;
  static bool configured[64] = {false};
  if (c->device < 0 || c->device >= 64 || !configured[c->device]) {
    cudaError_t e = cudaFuncSetAttribute(k_elem_f32<DIM, D, MODEL, E, G, DN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_check(e, "element kernel smem attribute");
    if (c->device >= 0 && c->device < 64) configured[c->device] = true;
  }
  const int64_t ntiles = (c->ne + kTile - 1) / kTile;
  const int grid = (int)(ntiles < kTileBlocks ? (ntiles > 0 ? ntiles : 1) : kTileBlocks);
  k_elem_f32<DIM, D, MODEL, E, G, DN><<<grid, kTile, smem, c->stream>>>(
      c->ne, A, c->u_df, c->eperm, mp, c->r32, dens, c->partials, node_partials, nb_node, c->counter, J,
      c->status);
  return cuda_check(cudaGetLastError(), "f32 element launch");
}

template <int DIM, int D, int MODEL>
fe_status eval32_t(fe_ctx* c, const double* v, double* J, double* dens, double* g, bool want_energy,
                   bool want_grad) {
  cudaStream_t s = c->stream;
  const ModelParams mp = model_params(c);
  const int nb_node = grid_for(c->nn, kMaxNodeBlocks);
  double* node_partials = c->partials + kMaxElemBlocks;
  prof_begin(c, kStagePrep);
  k_node_prep32<D, MODEL == FE_NEOHOOKE, DIM><<<nb_node, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b,
                                                                           c->u_df, node_partials, input_is_disp(c),
                                                                           input_is_disp(c) ? c->bX : 0.0);
  prof_end(c, kStagePrep);
  c->launches++;
  const bool E = want_energy, G = want_grad, Dn = dens != nullptr;
  if (c->ne > 0 || E) {
    prof_begin(c, kStageElem);
    fe_status es;
    if (E && G && Dn) es = launch_elem_f32<DIM, D, MODEL, true, true, true>(c, mp, dens, node_partials, nb_node, J);
    else if (E && G) es = launch_elem_f32<DIM, D, MODEL, true, true, false>(c, mp, dens, node_partials, nb_node, J);
    else if (E && Dn) es = launch_elem_f32<DIM, D, MODEL, true, false, true>(c, mp, dens, node_partials, nb_node, J);
    else if (E) es = launch_elem_f32<DIM, D, MODEL, true, false, false>(c, mp, dens, node_partials, nb_node, J);
    else if (G && Dn) es = launch_elem_f32<DIM, D, MODEL, false, true, true>(c, mp, dens, node_partials, nb_node, J);
    else if (G) es = launch_elem_f32<DIM, D, MODEL, false, true, false>(c, mp, dens, node_partials, nb_node, J);
    else es = launch_elem_f32<DIM, D, MODEL, false, false, true>(c, mp, dens, node_partials, nb_node, J);
    prof_end(c, kStageElem);
    c->launches++;
    if (es) return es;
  }
  if (G) {
    prof_begin(c, kStageGather);
    const fe_status gs = launch_gather_bulk<D, AccF32>(c, c->r32, g);
    prof_end(c, kStageGather);
    if (gs) return gs;
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
