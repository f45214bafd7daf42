// fe_eval_df64.cu -- energy and exact gradient in double-float arithmetic (FE_DF64).
//
// Same pipeline and data layout as the FP64 path (fe_eval_f64.cu) with every per-element
// floating-point operation done on pairs of floats (df64.cuh): GB300 has 64x more FP32 than
// FP64 throughput, and the double-float words carry about 48 bits, enough for the FP64
// tolerances (energy 1e-12 of its condition, gradient 1e-10 of its max norm).
//   k_node_prep_df  u = v - X in FP64, rounded to a double-float pair per component
//                   (32-byte node record in 3D), and the block partials of b.v in FP64
//   k_elem_df       F = I + sum_{l>=1} (u_l - u_0) grad(phi_l)^T (eq. Dv), W (eq. neoHook /
//                   eq. pLaplacian), dW/dF (Sec. 6.2), local forces to the CSR slots; the
//                   energy is accumulated as a double-float per thread, then in FP64 over
//                   the block and the grid (fixed order)
//   gather          per node: double-float sum of its CSR segment (warp-cooperative, bulk
//                   copies: gather_bulk.cuh), converted to FP64, - b
#include "df64.cuh"
#include "fe_internal.cuh"
#include "elem_df.cuh"
#include "gather_bulk.cuh"

namespace fe {
namespace {

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

template <int D, bool NH, int DIM>
__global__ void __launch_bounds__(kThreads) k_node_prep_df(int64_t nn, const double* __restrict__ v,
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
    const int64_t src = perm ? (int64_t)FE_CHK(perm[i], nn, kSiteNodePerm) : i;
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

template <int DIM, int D, int MODEL, bool ENERGY, bool GRAD, bool DENS>
__global__ void __launch_bounds__(kThreads) k_elem_df(
    int64_t ne, const int32_t* __restrict__ elems, const float2* __restrict__ dphi,
    const float2* __restrict__ vol, const float2* __restrict__ u, const int32_t* __restrict__ slot,
    const int32_t* __restrict__ eperm, ModelDF md, const LogEntry* __restrict__ log_tab,
    float2* __restrict__ r, double* __restrict__ dens, double* partials, const double* node_partials,
    int n_node_blocks, unsigned* counter, double* J, int* status) {
  constexpr int K = DIM + 1;
  __shared__ double sh[kThreads / 32];
  __shared__ LogEntry tab[kLogTable];
  if (MODEL == FE_NEOHOOKE && (ENERGY || DENS)) {
    for (int i = threadIdx.x; i < kLogTable; i += kThreads) tab[i] = log_tab[i];
    __syncthreads();
  }
  df acc = {0.f, 0.f};
  bool bad = false, inf_seen = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    df vT;
    const df W = elem_df_one<DIM, D, MODEL, ENERGY || DENS, GRAD>(e, ne, elems, dphi, vol, u, slot, md, tab, r,
                                                                 bad, vT);
    // W = +Inf (det F <= 0) would turn into NaN inside the double-float product: carry it aside
    if (ENERGY) {
      if (isinf(W.hi)) inf_seen = true;
      else acc = df_fma(vT, W, acc);
    }
    if (DENS) dens[eperm ? (int64_t)eperm[e] : e] = df_to_double(W);
  }
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) {
    const double t = block_sum(inf_seen ? CUDART_INF : df_to_double(acc), sh);
    finish_energy(t, partials, gridDim.x, node_partials, n_node_blocks, counter, J, sh);
  }
}

__global__ void k_to_df(int64_t n, const double* __restrict__ a, float2* __restrict__ o) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const df x = df_from_double(a[i]);
    o[i] = make_float2(x.hi, x.lo);
  }
}

// Logarithm table: c_i = kLogC0 + i/256, r_i = float(1/c_i), L_i = -log(r_i) (FP64 log).
__global__ void k_log_table(LogEntry* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kLogTable) return;
  const double c = (double)kLogC0 + (double)i / 256.0;
  const float r = (float)(1.0 / c);
  const df L = df_from_double(-log((double)r));
  tab[i] = LogEntry{r, L.hi, L.lo, 0.f};
}

__global__ void k_diag_log(int64_t n, const double* __restrict__ x, double* __restrict__ y,
                           const LogEntry* __restrict__ tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = df_to_double(df_log(df_from_double(x[i]), tab));
}

ModelDF model_df(const fe_ctx* c) {
  ModelDF m;
  auto split = [](double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
  };
  m.C1 = split(c->C1);
  m.D1 = split(c->D1);
  m.twoC1 = split(2.0 * c->C1);
  m.twoD1 = split(2.0 * c->D1);
  m.negTwoC1 = split(-2.0 * c->C1);
  m.p = c->p;
  m.pcase = (c->p == 2.0) ? 2 : (c->p == 3.0) ? 3 : (c->p == 4.0) ? 4 : (c->p == 1.5) ? 15 : 0;
  return m;
}

template <int DIM, int D, int MODEL>
fe_status evaldf_t(fe_ctx* c, const double* v, double* J, double* dens, double* g, bool want_energy,
                   bool want_grad) {
  cudaStream_t s = c->stream;
  const ModelDF md = model_df(c);
  const int nb_node = grid_for(c->nn, kMaxNodeBlocks);
  const int nb_elem = grid_for(c->ne, kMaxElemBlocks);
  double* node_partials = c->partials + kMaxElemBlocks;
  prof_begin(c, kStagePrep);
  k_node_prep_df<D, MODEL == FE_NEOHOOKE, DIM><<<nb_node, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b,
                                                                            c->u_df, node_partials, input_is_disp(c),
                                                                            input_is_disp(c) ? c->bX : 0.0);
  prof_end(c, kStagePrep);
  c->launches++;
  const bool E = want_energy, G = want_grad, Dn = dens != nullptr;
#define FE_ELEMDF(EN, GR, DE)                                                                             \
  k_elem_df<DIM, D, MODEL, EN, GR, DE><<<nb_elem, kThreads, 0, s>>>(                                      \
      c->ne, c->elems, c->dphi_df, c->vol_df, c->u_df, c->slot, c->eperm, md, c->log_tab, c->r_df, dens,   \
      c->partials, node_partials, nb_node, c->counter, J, c->status)
  if (c->ne > 0 || E) {
    prof_begin(c, kStageElem);
    if (E && G && Dn) FE_ELEMDF(true, true, true);
    else if (E && G) FE_ELEMDF(true, true, false);
    else if (E && Dn) FE_ELEMDF(true, false, true);
    else if (E) FE_ELEMDF(true, false, false);
    else if (G && Dn) FE_ELEMDF(false, true, true);
    else if (G) FE_ELEMDF(false, true, false);
    else FE_ELEMDF(false, false, true);
    prof_end(c, kStageElem);
    c->launches++;
  }
#undef FE_ELEMDF
  if (G) {
    prof_begin(c, kStageGather);
    const fe_status gs = launch_gather_bulk<D, AccDF>(c, c->r_df, g);
    prof_end(c, kStageGather);
    if (gs) return gs;
    c->launches++;
  }
  return cuda_check(cudaGetLastError(), "eval df64 launch");
}

}  // namespace

fe_status launch_precompute_df(fe_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t nd = c->ne * c->dim * c->dim;
  if (c->ne > 0) {
    k_to_df<<<grid_for(nd, 4 * kMaxElemBlocks), kThreads, 0, s>>>(nd, c->dphi, c->dphi_df);
    k_to_df<<<grid_for(c->ne, 4 * kMaxElemBlocks), kThreads, 0, s>>>(c->ne, c->vol, c->vol_df);
    c->launches += 2;
  }
  k_log_table<<<1, kLogTable, 0, s>>>(c->log_tab);
  c->launches++;
  return cuda_check(cudaGetLastError(), "precompute df64 launch");
}

fe_status launch_eval_df64(fe_ctx* c, const double* v, double* J, double* dens, double* g,
                           bool want_energy, bool want_grad) {
  if (c->model == FE_NEOHOOKE) {
    if (c->dim == 2) return evaldf_t<2, 2, FE_NEOHOOKE>(c, v, J, dens, g, want_energy, want_grad);
    return evaldf_t<3, 3, FE_NEOHOOKE>(c, v, J, dens, g, want_energy, want_grad);
  }
  if (c->dim == 2) return evaldf_t<2, 1, FE_PLAPLACE>(c, v, J, dens, g, want_energy, want_grad);
  return evaldf_t<3, 1, FE_PLAPLACE>(c, v, J, dens, g, want_energy, want_grad);
}

fe_status launch_diag_df_log(const LogEntry* tab, const double* x, double* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return FE_OK;
  k_diag_log<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, x, y, tab);
  return cuda_check(cudaGetLastError(), "diag log launch");
}

fe_status launch_log_table(LogEntry* tab, cudaStream_t s) {
  k_log_table<<<1, kLogTable, 0, s>>>(tab);
  return cuda_check(cudaGetLastError(), "log table launch");
}

}  // namespace fe
