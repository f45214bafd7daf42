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

__device__ __forceinline__ df ld_df(const float2* __restrict__ p, int64_t i) {
  const float2 a = __ldg(p + i);
  return {a.x, a.y};
}

// Node record of the double-float displacement: D pairs, padded to 4 pairs in 3D.
template <int D>
__device__ __forceinline__ void load_u_df(const float2* __restrict__ u, int32_t n, df* out) {
  if (D == 1) {
    out[0] = ld_df(u, n);
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

// Sum of squares of N double-floats: exact leading products, TwoSum chain.
template <int N>
__device__ __forceinline__ df df_sumsq(const df* x) {
  float s = fmul(x[0].hi, x[0].hi);
  float e = fmaf(x[0].hi, x[0].hi, -s);
  e = fmaf(fmul(2.f, x[0].hi), x[0].lo, e);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const float p = fmul(x[i].hi, x[i].hi);
    e = fadd(e, fmaf(x[i].hi, x[i].hi, -p));
    e = fmaf(fmul(2.f, x[i].hi), x[i].lo, e);
    const df t = two_sum(s, p);
    s = t.hi;
    e = fadd(e, t.lo);
  }
  return fast_two_sum(s, e);
}

// Model constants as double-floats.
struct ModelDF {
  df C1, D1, twoC1, twoD1, negTwoC1;
  int pcase;     // p-Laplacian: 2, 3, 4, 15 (p = 1.5) in double-float; 0 = general p (FP64)
  double p;
};

// General p-Laplacian exponent: W = s^(p/2)/p and the coefficient s^((p-2)/2) in FP64.
__device__ __noinline__ void plap_general_f64(double s, double p, double* W, double* coef) {
  *W = s > 0.0 ? pow(s, 0.5 * p) / p : 0.0;
  *coef = s > 0.0 ? pow(s, 0.5 * (p - 2.0)) : 0.0;
}

template <int D, bool NH, int DIM>
__global__ void __launch_bounds__(kThreads) k_node_prep_df(int64_t nn, const double* __restrict__ v,
                                                           const double* __restrict__ X,
                                                           const int32_t* __restrict__ perm,
                                                           const double* __restrict__ b,
                                                           float2* __restrict__ u,
                                                           double* __restrict__ node_partials) {
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
      w[j] = df_from_double(NH ? vj - X[i * DIM + j] : vj);
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
  if (threadIdx.x == 0) node_partials[blockIdx.x] = dot;
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
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    df ul[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) load_u_df<D>(u, __ldg(elems + (int64_t)l * ne + e), ul[l]);
    df g[DIM][DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = ld_df(dphi, ((int64_t)l * DIM + m) * ne + e);
    const df vT = ld_df(vol, e);
    // H_jm = sum_{l>=1} (u_l - u_0)_j dphi_lm
    df H[D][DIM];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      df a[DIM];
#pragma unroll
      for (int l = 0; l < DIM; ++l) a[l] = df_sub(ul[l + 1][j], ul[0][j]);
#pragma unroll
      for (int m = 0; m < DIM; ++m)
        H[j][m] = (DIM == 3) ? df_dot3(a[0], g[0][m], a[1], g[1][m], a[DIM - 1], g[DIM - 1][m])
                             : df_dot2(a[0], g[0][m], a[DIM - 1], g[DIM - 1][m]);
    }
    df W = {0.f, 0.f};
    df P[D][DIM];
    if (MODEL == FE_NEOHOOKE) {
      df F[DIM][DIM], C[DIM][DIM], det;
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) F[j][m] = (j == m) ? df_add_f(H[j][m], 1.0f) : H[j][m];
      if (DIM == 3) {
        C[0][0] = df_det2(F[1][1], F[2][2], F[1][2], F[2][1]);
        C[0][1] = df_det2(F[1][2], F[2][0], F[1][0], F[2][2]);
        C[0][2] = df_det2(F[1][0], F[2][1], F[1][1], F[2][0]);
        det = df_dot3(F[0][0], C[0][0], F[0][1], C[0][1], F[0][DIM - 1], C[0][DIM - 1]);
        if (GRAD) {
          C[1][0] = df_det2(F[0][2], F[2][1], F[0][1], F[2][2]);
          C[1][1] = df_det2(F[0][0], F[2][2], F[0][2], F[2][0]);
          C[1][2] = df_det2(F[0][1], F[2][0], F[0][0], F[2][1]);
          C[2][0] = df_det2(F[0][1], F[1][2], F[0][2], F[1][1]);
          C[2][1] = df_det2(F[0][2], F[1][0], F[0][0], F[1][2]);
          C[2][2] = df_det2(F[0][0], F[1][1], F[0][1], F[1][0]);
        }
      } else {
        C[0][0] = F[1][1];
        C[0][1] = df_neg(F[1][0]);
        C[1][0] = df_neg(F[0][1]);
        C[1][1] = F[0][0];
        det = df_det2(F[0][0], F[1][1], F[0][1], F[1][0]);
      }
      const bool ebad = !(det.hi > 0.f);
      const df delta = df_add_f(det, -1.0f);
      if (ENERGY || DENS) {
        // W = C1 (I1 - dim - 2 log det F) + D1 (det F - 1)^2, with I1 - dim = 2 tr H + |H|^2
        df tr = H[0][0];
#pragma unroll
        for (int j = 1; j < DIM; ++j) tr = df_add(tr, H[j][j]);
        const df hsq = df_sumsq<D * DIM>(&H[0][0]);
        const df lg = df_log(ebad ? df{1.f, 0.f} : det, tab);
        const df br = df_add(df_add(df_scale(tr, 2.f), hsq), df_scale(lg, -2.f));
        W = df_dot2(md.C1, br, md.D1, df_sqr(delta));
        if (ebad) W = {CUDART_INF_F, 0.f};
      }
      if (GRAD) {
        // dW/dF = 2 C1 F + (2 D1 (det F - 1) - 2 C1 / det F) cof F, times |T|
        const df rJ = df_rcp(det);
        const df a = df_mul(md.twoC1, vT);
        const df c = df_mul(vT, df_dot2(md.twoD1, delta, md.negTwoC1, rJ));
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int m = 0; m < DIM; ++m) P[j][m] = df_dot2(a, F[j][m], c, C[j][m]);
      }
      bad |= ebad;
    } else {
      const df s = df_sumsq<DIM>(&H[0][0]);
      df coef = {1.f, 0.f};
      if (md.pcase == 2) {
        W = df_scale(s, 0.5f);
      } else if (md.pcase == 3) {
        coef = df_sqrt(s);
        W = df_mul(df_mul(s, coef), df{0x1.555556p-2f, -0x1.555556p-27f});
      } else if (md.pcase == 4) {
        coef = s;
        W = df_scale(df_sqr(s), 0.25f);
      } else if (md.pcase == 15) {
        const df q = df_sqrt(s), qq = df_sqrt(q);                // s^(1/2), s^(1/4)
        W = df_mul(df_mul(q, qq), df{0x1.555556p-1f, -0x1.555556p-26f});   // s^(3/4) / 1.5
        coef = (qq.hi > 0.f) ? df_rcp(qq) : df{0.f, 0.f};        // s^(-1/4)
      } else {
        double Wd, cd;
        plap_general_f64(df_to_double(s), md.p, &Wd, &cd);
        W = df_from_double(Wd);
        coef = df_from_double(cd);
      }
      if (GRAD) {
        const df c = df_mul(vT, coef);
#pragma unroll
        for (int m = 0; m < DIM; ++m) P[0][m] = df_mul(c, H[0][m]);
      }
    }
    if (ENERGY) acc = df_fma(vT, W, acc);
    if (DENS) dens[eperm ? (int64_t)eperm[e] : e] = df_to_double(W);
    if (GRAD) {
      df r0[D];
#pragma unroll
      for (int j = 0; j < D; ++j) r0[j] = {0.f, 0.f};
#pragma unroll
      for (int l = 1; l <= DIM; ++l) {
        const int64_t q = __ldg(slot + (int64_t)l * ne + e);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const df s = (DIM == 3) ? df_dot3(P[j][0], g[l - 1][0], P[j][1], g[l - 1][1], P[j][DIM - 1], g[l - 1][DIM - 1])
                                  : df_dot2(P[j][0], g[l - 1][0], P[j][DIM - 1], g[l - 1][DIM - 1]);
          r[q * D + j] = make_float2(s.hi, s.lo);
          r0[j] = df_sub(r0[j], s);
        }
      }
      const int64_t q0 = __ldg(slot + e);
#pragma unroll
      for (int j = 0; j < D; ++j) r[q0 * D + j] = make_float2(r0[j].hi, r0[j].lo);
    }
  }
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) {
    const double t = block_sum(df_to_double(acc), sh);
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
  k_node_prep_df<D, MODEL == FE_NEOHOOKE, DIM><<<nb_node, kThreads, 0, s>>>(c->nn, v, c->X, c->perm, c->b,
                                                                            c->u_df, node_partials);
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
