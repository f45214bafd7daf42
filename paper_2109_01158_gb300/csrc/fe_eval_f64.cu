// fe_eval_f64.cu -- FP64 evaluation of the energy J(v) = sum |T| W(F_T) - b.v, its exact
// gradient and the patch-local central-difference gradient (Sec. 5, 6.1 and 6.2).
//
// Pipeline of one call (all on the context stream):
//   k_node_prep   v (caller order) -> u (device order): u = v - X for Neo-Hookean
//                 (displacement form of F = grad v; u = v when the caller passes
//                 displacements), u = v for the p-Laplacian; also the block partials of b.v.
//   k_elem_f64    one thread per element (grid-stride, fixed grid): gathers u at the
//                 dim+1 vertices, forms F = I + sum_{l>=1} (u_l - u_0) grad(phi_l)^T (the
//                 same matrix as eq. Dv because sum_l grad(phi_l) = 0 and
//                 sum_l X_l grad(phi_l)^T = I), evaluates W (and dW/dF), accumulates
//                 |T| W, and writes the local forces r_{T,l} = |T| dW/dF grad(phi_l) to the
//                 CSR position of (T, l); the last block to finish reduces the partials.
//   k_gather_bulk one lane per node, 32-node patch blocks staged in shared memory by bulk
//                 copies: g_i = sum of its CSR segment - b_i (0 on Dirichlet dofs), written
//                 in the caller's dof order.
// Every reduction has a fixed order, so results are bitwise reproducible.
#include "fe_internal.cuh"
#include "gather_bulk.cuh"
#include "phi_f64.cuh"  // phi(x) = x - log(1 + x) and 1/(1 + x) from the breakpoint table
#include "density_f64.cuh"  // W of eqs. neoHook / pLaplacian in FP64

namespace fe {
namespace {

// ---- block reduction helpers -----------------------------------------------------------

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Sum over the block in a fixed tree; the result is valid in thread 0.
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

// The block that finishes last sums the element partials and the b.v partials in a fixed
// order and writes J = sum |T| W - b.v.
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

// Load the displacement of one node: stride DP doubles (16-byte aligned for DP >= 2).
template <int D>
__device__ __forceinline__ void load_u(const double* __restrict__ u, int32_t n, double* out) {
  if (D == 1) {
    out[0] = __ldg(u + n);
  } else if (D == 2) {
    double2 a = __ldg(reinterpret_cast<const double2*>(u) + n);
    out[0] = a.x;
    out[1] = a.y;
  } else {
    const double2* p = reinterpret_cast<const double2*>(u) + 2 * (int64_t)n;
    double2 a = __ldg(p), b = __ldg(p + 1);
    out[0] = a.x;
    out[1] = a.y;
    out[2] = b.x;
  }
}

template <int DIM>
struct Mat64 {
  double m[DIM][DIM];
};

// |T| dW/dF near F = I without O(1) terms: 2 C1 (H - L) + 2 delta (D1 + C1 / det F) cof F with
// L = cof F - I, whose diagonal L_jj is formed from H (X0 = L_00 from the caller).  Out of
// line: the common path keeps the registers and code of the plain form.
template <int DIM>
static __device__ __noinline__ Mat64<DIM> nh_stress_small_f64(Mat64<DIM> H, Mat64<DIM> C, double X0, double delta,
                                                               double det, double a, double vT, double C1,
                                                               double D1) {
  double Ld[DIM];
  if constexpr (DIM == 3) {
    Ld[0] = X0;
    Ld[1] = H.m[0][0] + H.m[2][2] + (H.m[0][0] * H.m[2][2] - H.m[0][2] * H.m[2][0]);
    Ld[2] = H.m[0][0] + H.m[1][1] + (H.m[0][0] * H.m[1][1] - H.m[0][1] * H.m[1][0]);
  } else {
    Ld[0] = H.m[1][1];
    Ld[1] = H.m[0][0];
  }
  const double cp = 2.0 * vT * delta * (D1 + C1 / det);
  Mat64<DIM> P;
#pragma unroll
  for (int j = 0; j < DIM; ++j)
#pragma unroll
    for (int m = 0; m < DIM; ++m) P.m[j][m] = fma(a, H.m[j][m] - (j == m ? Ld[j] : C.m[j][m]), cp * C.m[j][m]);
  return P;
}

// ---- kernels ------------------------------------------------------------------------------

template <int D, bool NH, int DIM>
__global__ void __launch_bounds__(kThreads) k_node_prep(int64_t nn, const double* __restrict__ v,
                                                        const double* __restrict__ X,
                                                        const int32_t* __restrict__ perm,
                                                        const double* __restrict__ b,
                                                        double* __restrict__ u,
                                                        double* __restrict__ node_partials, bool disp,
    double shift) {
  __shared__ double sh[kThreads / 32];
  constexpr int DP = D == 3 ? 4 : D;
  double dot = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    const int64_t src = perm ? (int64_t)FE_CHK(perm[i], nn, kSiteNodePerm) : i;
    double w[DP];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const double vj = v[src * D + j];
      dot += b[i * D + j] * vj;
      w[j] = (NH && !disp) ? vj - X[i * DIM + j] : vj;
    }
    if (DP == 4) w[3] = 0.0;
    if (DP == 1) {
      u[i] = w[0];
    } else {
      double2* o = reinterpret_cast<double2*>(u) + i * (DP / 2);
      o[0] = make_double2(w[0], w[1]);
      if (DP == 4) o[1] = make_double2(w[2], w[3]);
    }
  }
  dot = block_sum(dot, sh);
  // block 0 adds b.X when v is a displacement (then dot sums b.u)
  if (threadIdx.x == 0) node_partials[blockIdx.x] = (blockIdx.x == 0 && disp) ? dot + shift : dot;
}

// Element kernel: energy partials, densities, and/or local forces.
template <int DIM, int D, int MODEL, bool ENERGY, bool GRAD, bool DENS>
__global__ void __launch_bounds__(kThreads) k_elem_f64(
    int64_t ne, const int32_t* __restrict__ elems, const double* __restrict__ dphi,
    const double* __restrict__ vol, const double* __restrict__ u, const int32_t* __restrict__ slot,
    const int32_t* __restrict__ eperm, ModelParams mp, double* __restrict__ r,
    double* __restrict__ dens, double* partials, const double* node_partials, int n_node_blocks,
    unsigned* counter, double* J, int* status) {
  constexpr int K = DIM + 1;
  __shared__ double sh[kThreads / 32];
  double acc = 0.0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    double ul[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) load_u<D>(u, FE_CHK(__ldg(elems + (int64_t)l * ne + e), mp.nn, kSiteElemNode), ul[l]);
    double g[DIM][DIM];  // grad(phi_l), l = 1..DIM
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = __ldg(dphi + ((int64_t)l * DIM + m) * ne + e);
    const double vT = __ldg(vol + e);
    // H_jm = sum_{l>=1} (u_l - u_0)_j dphi_lm
    double H[D][DIM];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double a[DIM];
#pragma unroll
      for (int l = 0; l < DIM; ++l) a[l] = ul[l + 1][j] - ul[0][j];
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        double s = a[0] * g[0][m];
#pragma unroll
        for (int l = 1; l < DIM; ++l) s = fma(a[l], g[l][m], s);
        H[j][m] = s;
      }
    }
    double W = 0.0;
    double P[D][DIM];
    if (MODEL == FE_NEOHOOKE) {
      // Displacement form of eq. neoHook with F = I + H (same value, no cancellation of O(1)
      // terms): delta = det F - 1 = tr H + q, q = i2(H) + det H, and
      //   I1 - dim - 2 log det F = |H|^2 - 2 q + 2 phi(delta),  phi(x) = x - log(1 + x).
      double Fm[DIM][DIM], Cm[DIM][DIM], q, tr = H[0][0], hsq = 0.0, X0 = 0.0;
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        if (j > 0) tr += H[j][j];
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          Fm[j][m] = (j == m) ? 1.0 + H[j][m] : H[j][m];
          hsq = fma(H[j][m], H[j][m], hsq);
        }
      }
      if (DIM == 3) {
        const double M00 = H[1][1] * H[DIM - 1][DIM - 1] - H[1][DIM - 1] * H[DIM - 1][1];
        const double X = H[1][1] + H[DIM - 1][DIM - 1] + M00;
        X0 = X;
        Cm[0][0] = 1.0 + X;
        Cm[0][1] = Fm[1][2] * Fm[2][0] - Fm[1][0] * Fm[2][2];
        Cm[0][2] = Fm[1][0] * Fm[2][1] - Fm[1][1] * Fm[2][0];
        Cm[1][0] = Fm[0][2] * Fm[2][1] - Fm[0][1] * Fm[2][2];
        Cm[1][1] = Fm[0][0] * Fm[2][2] - Fm[0][2] * Fm[2][0];
        Cm[1][2] = Fm[0][1] * Fm[2][0] - Fm[0][0] * Fm[2][1];
        Cm[2][0] = Fm[0][1] * Fm[1][2] - Fm[0][2] * Fm[1][1];
        Cm[2][1] = Fm[0][2] * Fm[1][0] - Fm[0][0] * Fm[1][2];
        Cm[2][2] = Fm[0][0] * Fm[1][1] - Fm[0][1] * Fm[1][0];
        q = M00 + H[0][0] * X + H[0][1] * Cm[0][1] + H[0][DIM - 1] * Cm[0][DIM - 1];
      } else {
        Cm[0][0] = Fm[1][1];
        Cm[0][1] = -Fm[1][0];
        Cm[1][0] = -Fm[0][1];
        Cm[1][1] = Fm[0][0];
        q = H[0][0] * H[1][1] - H[0][1] * H[1][0];
      }
      const double delta = tr + q;
      const double det = 1.0 + delta;
      double rdet = 0.0;   // 1 / det F
      if (!(det > 0.0)) {
        bad = true;
        W = CUDART_INF;
      } else if (ENERGY || DENS) {
        const double ph = GRAD ? phi_rcp_f64(delta, &rdet) : phi_f64(delta);
        W = mp.C1 * (hsq - 2.0 * q + 2.0 * ph) + mp.D1 * delta * delta;
      }
      if (GRAD && !(ENERGY || DENS)) rdet = rcp1p_f64(delta);
      if (GRAD) {
        // dW/dF = 2 C1 F + (2 D1 delta - 2 C1 / det F) cof F.  Near F = I its two terms cancel
        // to O(|H|), leaving a relative error of about u / |H|; a warp with any |H|^2 < 1e-4
        // uses instead the same value as
        //   2 C1 (H - L) + 2 delta (D1 + C1 / det F) cof F,   L = cof F - I,
        // whose diagonal L_jj is formed from H without the 1 (no O(1) term left).
        const double a = mp.twoC1 * vT;
        // hsq < 1e-4 by the bit pattern (hsq >= 0): an integer compare
        if (__any_sync(__activemask(), __double_as_longlong(hsq) < 0x3F1A36E2EB1C432DLL)) {
          Mat64<DIM> h, cf;
#pragma unroll
          for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int m = 0; m < DIM; ++m) {
              h.m[j][m] = H[j][m];
              cf.m[j][m] = Cm[j][m];
            }
          const Mat64<DIM> p = nh_stress_small_f64<DIM>(h, cf, X0, delta, det, a, vT, mp.C1, mp.D1);
#pragma unroll
          for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int m = 0; m < DIM; ++m) P[j][m] = p.m[j][m];
        } else {
          const double c = vT * fma(mp.twoD1, delta, -mp.twoC1 * rdet);
#pragma unroll
          for (int j = 0; j < D; ++j)
#pragma unroll
            for (int m = 0; m < DIM; ++m) P[j][m] = fma(a, Fm[j][m], c * Cm[j][m]);
        }
      }
    } else if constexpr (MODEL == FE_PLAPLACE_LP) {
      // W = (1/p) sum_m |H_m|^p, dW/dH_m = |H_m|^(p-2) H_m
      double sp = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        double ap, ap2;
        plap_lp_terms(H[0][m], mp, &ap, &ap2);
        sp += ap;
        if (GRAD) P[0][m] = vT * ap2 * H[0][m];
      }
      if (ENERGY || DENS) W = sp / mp.p;
    } else {
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) s = fma(H[0][m], H[0][m], s);
      if (ENERGY || DENS) W = plap_density(s, mp);
      if (GRAD) {
        const double c = vT * plap_coef(s, mp);
#pragma unroll
        for (int m = 0; m < DIM; ++m) P[0][m] = c * H[0][m];
      }
    }
    if (ENERGY) acc = fma(vT, W, acc);
    if (DENS) dens[eperm ? (int64_t)FE_CHK(eperm[e], ne, kSiteElemPerm) : e] = W;
    if (GRAD) {
      // r_l = |T| P grad(phi_l) for l >= 1, r_0 = -sum_{l>=1} r_l (grad(phi_0) = -sum grad(phi_l))
      double r0[D];
#pragma unroll
      for (int l = 1; l <= DIM; ++l) {
        const int64_t q = FE_CHK(__ldg(slot + (int64_t)l * ne + e), ne * K, kSiteElemSlot);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double s = P[j][0] * g[l - 1][0];
#pragma unroll
          for (int m = 1; m < DIM; ++m) s = fma(P[j][m], g[l - 1][m], s);
          r[q * D + j] = s;
          r0[j] = (l == 1) ? -s : r0[j] - s;   // (the first term needs no addition)
        }
      }
      const int64_t q0 = FE_CHK(__ldg(slot + e), ne * K, kSiteElemSlot);
#pragma unroll
      for (int j = 0; j < D; ++j) r[q0 * D + j] = r0[j];
    }
  }
  if (bad) atomicOr(status, kStatusDomain);
  if (ENERGY) {
    acc = block_sum(acc, sh);
    finish_energy(acc, partials, gridDim.x, node_partials, n_node_blocks, counter, J, sh);
  }
}

// ---- central differences over patches (Sec. 6.1) ------------------------------------------

// W at F_T with row j recomputed from nodal values whose entry (local lc, component j) is
// shifted by delta (the GG layer of component j).  ul: element nodal values.
template <int DIM, int D, int MODEL>
__device__ __forceinline__ double fd_density(double ul[DIM + 1][D], const double g[DIM][DIM],
                                             const double H[D][DIM], int lc, int j, double delta,
                                             const ModelParams& mp, bool& bad) {
  double row[DIM];
  double a[DIM];
  const double u0 = (lc == 0) ? ul[0][j] + delta : ul[0][j];
#pragma unroll
  for (int l = 0; l < DIM; ++l) a[l] = ((lc == l + 1) ? ul[l + 1][j] + delta : ul[l + 1][j]) - u0;
#pragma unroll
  for (int m = 0; m < DIM; ++m) {
    double s = a[0] * g[0][m];
#pragma unroll
    for (int l = 1; l < DIM; ++l) s = fma(a[l], g[l][m], s);
    row[m] = s;
  }
  if constexpr (MODEL == FE_NEOHOOKE) {
    double Hx[DIM][DIM];
#pragma unroll
    for (int jj = 0; jj < DIM; ++jj)
#pragma unroll
      for (int m = 0; m < DIM; ++m) Hx[jj][m] = (jj == j) ? row[m] : H[jj][m];
    return nh_density_disp<DIM>(Hx, mp, bad);
  } else if constexpr (MODEL == FE_PLAPLACE_LP) {
    double sp = 0.0;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      double ap, ap2;
      plap_lp_terms(row[m], mp, &ap, &ap2);
      sp += ap;
    }
    return sp / mp.p;
  } else {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < DIM; ++m) s = fma(row[m], row[m], s);
    return plap_density(s, mp);
  }
}

template <int DIM, int D>
__device__ __forceinline__ void element_state(int64_t e, int64_t ne, const int32_t* __restrict__ elems,
                                              const double* __restrict__ dphi,
                                              const double* __restrict__ u, double ul[DIM + 1][D],
                                              double g[DIM][DIM], double H[D][DIM]) {
#pragma unroll
  for (int l = 0; l <= DIM; ++l) load_u<D>(u, __ldg(elems + (int64_t)l * ne + e), ul[l]);
#pragma unroll
  for (int l = 0; l < DIM; ++l)
#pragma unroll
    for (int m = 0; m < DIM; ++m) g[l][m] = __ldg(dphi + ((int64_t)l * DIM + m) * ne + e);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double a[DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l) a[l] = ul[l + 1][j] - ul[0][j];
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      double s = a[0] * g[0][m];
#pragma unroll
      for (int l = 1; l < DIM; ++l) s = fma(a[l], g[l][m], s);
      H[j][m] = s;
    }
  }
}

// Full mode: |T| W(F^{+-}) for every (element, local node, component), written to the CSR
// position of (T, l): plus values in rp, minus values in rm.
template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_elem_fd_f64(int64_t ne, const int32_t* __restrict__ elems,
                                                          const double* __restrict__ dphi,
                                                          const double* __restrict__ vol,
                                                          const double* __restrict__ u,
                                                          const int32_t* __restrict__ slot, ModelParams mp,
                                                          double eps, double* __restrict__ rp,
                                                          double* __restrict__ rm, int* status) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    double ul[DIM + 1][D], g[DIM][DIM], H[D][DIM];
    element_state<DIM, D>(e, ne, elems, dphi, u, ul, g, H);
    const double vT = __ldg(vol + e);
#pragma unroll
    for (int lc = 0; lc <= DIM; ++lc) {
      const int64_t q = __ldg(slot + (int64_t)lc * ne + e);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        rp[q * D + j] = vT * fd_density<DIM, D, MODEL>(ul, g, H, lc, j, eps, mp, bad);
        rm[q * D + j] = vT * fd_density<DIM, D, MODEL>(ul, g, H, lc, j, -eps, mp, bad);
      }
    }
  }
  if (bad) atomicOr(status, kStatusDomain);
}

// Full mode, Neo-Hookean: the perturbation of row j of F by +-eps grad(phi_l) (the GG layer of
// the dof (l, j), with grad(phi_0) = -sum_l grad(phi_l)) changes the terms of the displacement
// form exactly as follows (det F is linear in each row, |H|^2 is quadratic):
//   q  -> q + e (cof F - I)_j . grad(phi_l),   tr H -> tr H + e grad(phi_l)_j,
//   |H|^2 -> |H|^2 + e (2 H_j . grad(phi_l) + e |grad(phi_l)|^2),   delta = tr H + q,
// so each of the 2 (dim + 1) dim densities costs a few operations and one phi instead of a
// full density.  (cof F - I) is formed from H without the 1 on its diagonal.  Writes
// |T| (W+ - W-) / (2 eps) to the CSR position of (T, l), which the bulk gather sums over the
// patch (the central difference of eq. CD restricted to the patch, eq. CDS).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_elem_fd_nh_f64(int64_t ne, const int32_t* __restrict__ elems,
                                                             const double* __restrict__ dphi,
                                                             const double* __restrict__ vol,
                                                             const double* __restrict__ u,
                                                             const int32_t* __restrict__ slot, ModelParams mp,
                                                             double eps, double* __restrict__ r, int* status) {
  bool bad = false;
  const double inv2e = 1.0 / (2.0 * eps);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    double ul[DIM + 1][DIM], g[DIM][DIM], H[DIM][DIM];
    element_state<DIM, DIM>(e, ne, elems, dphi, u, ul, g, H);
    const double vT = __ldg(vol + e);
    double tr = H[0][0], hsq = 0.0, q, L[DIM][DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      if (j > 0) tr += H[j][j];
#pragma unroll
      for (int m = 0; m < DIM; ++m) hsq = fma(H[j][m], H[j][m], hsq);
    }
    if constexpr (DIM == 3) {
      L[0][0] = H[1][1] + H[2][2] + (H[1][1] * H[2][2] - H[1][2] * H[2][1]);
      L[1][1] = H[0][0] + H[2][2] + (H[0][0] * H[2][2] - H[0][2] * H[2][0]);
      L[2][2] = H[0][0] + H[1][1] + (H[0][0] * H[1][1] - H[0][1] * H[1][0]);
      L[0][1] = H[1][2] * H[2][0] - H[1][0] * (1.0 + H[2][2]);
      L[0][2] = H[1][0] * H[2][1] - (1.0 + H[1][1]) * H[2][0];
      L[1][0] = H[0][2] * H[2][1] - H[0][1] * (1.0 + H[2][2]);
      L[1][2] = H[0][1] * H[2][0] - (1.0 + H[0][0]) * H[2][1];
      L[2][0] = H[0][1] * H[1][2] - H[0][2] * (1.0 + H[1][1]);
      L[2][1] = H[0][2] * H[1][0] - (1.0 + H[0][0]) * H[1][2];
      const double M00 = H[1][1] * H[2][2] - H[1][2] * H[2][1];
      q = M00 + H[0][0] * L[0][0] + H[0][1] * L[0][1] + H[0][2] * L[0][2];
    } else {
      L[0][0] = H[1][1];
      L[1][1] = H[0][0];
      L[0][1] = -H[1][0];
      L[1][0] = -H[0][1];
      q = H[0][0] * H[1][1] - H[0][1] * H[1][0];
    }
#pragma unroll
    for (int lc = 0; lc <= DIM; ++lc) {
      double gv[DIM];
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        if (lc > 0) {
          gv[m] = g[lc - 1][m];
        } else {
          double t = 0.0;
#pragma unroll
          for (int l = 0; l < DIM; ++l) t -= g[l][m];
          gv[m] = t;
        }
      }
      double gg = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) gg = fma(gv[m], gv[m], gg);
      const int64_t qs = __ldg(slot + (int64_t)lc * ne + e);
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        double lg = 0.0, hg = 0.0;
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          lg = fma(L[j][m], gv[m], lg);
          hg = fma(H[j][m], gv[m], hg);
        }
        double Wpm[2];
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
          const double ee = sgn == 0 ? eps : -eps;
          const double qx = fma(ee, lg, q);
          const double dl = fma(ee, gv[j], tr) + qx;
          const double hs = fma(ee, fma(ee, gg, 2.0 * hg), hsq);
          if (!(1.0 + dl > 0.0)) {
            bad = true;
            Wpm[sgn] = CUDART_INF;
          } else {
            Wpm[sgn] = mp.C1 * (hs - 2.0 * qx + 2.0 * phi_f64(dl)) + mp.D1 * dl * dl;
          }
        }
        r[qs * DIM + j] = (vT * Wpm[0] - vT * Wpm[1]) * inv2e;
      }
    }
  }
  if (bad) atomicOr(status, kStatusDomain);
}

template <int D>
__global__ void __launch_bounds__(kThreads) k_gather_fd(int64_t nn, const int32_t* __restrict__ row_ptr,
                                                        const double* __restrict__ rp,
                                                        const double* __restrict__ rm, double eps,
                                                        const double* __restrict__ b,
                                                        const uint8_t* __restrict__ dir,
                                                        const int32_t* __restrict__ perm,
                                                        double* __restrict__ g) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    double sp[D], sm[D];
#pragma unroll
    for (int j = 0; j < D; ++j) sp[j] = sm[j] = 0.0;
    const int32_t q1 = row_ptr[i + 1];
    for (int32_t q = row_ptr[i]; q < q1; ++q)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        sp[j] += rp[(int64_t)q * D + j];
        sm[j] += rm[(int64_t)q * D + j];
      }
    const int64_t dst = perm ? (int64_t)perm[i] : i;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const double val = (sp[j] - sm[j]) / (2.0 * eps) - b[i * D + j];
      g[dst * D + j] = dir[i * D + j] ? 0.0 : val;
    }
  }
}

// Subset mode: one thread per requested dof walks the patch of its node.
template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_fd_subset(int64_t ndofs, const int64_t* __restrict__ dofs,
                                                        const int32_t* __restrict__ iperm, int64_t nn,
                                                        int64_t ne, const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ ent,
                                                        const int32_t* __restrict__ elems,
                                                        const double* __restrict__ dphi,
                                                        const double* __restrict__ vol,
                                                        const double* __restrict__ u,
                                                        const double* __restrict__ b,
                                                        const uint8_t* __restrict__ dir, ModelParams mp,
                                                        double eps, double* __restrict__ g,
                                                        int* status) {
  constexpr int K = DIM + 1;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ndofs; t += stride) {
    const int64_t n = dofs[t];
    if (n < 0 || n >= nn * D) {
      g[t] = CUDART_NAN;
      continue;
    }
    const int64_t iu = n / D;
    const int j = (int)(n % D);
    const int64_t i = iperm ? (int64_t)iperm[iu] : iu;
    if (dir[i * D + j]) {
      g[t] = 0.0;
      continue;
    }
    double sp = 0.0, sm = 0.0;
    for (int32_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      const int32_t en = ent[q];
      const int64_t e = en / K;
      const int lc = en % K;
      double ul[DIM + 1][D], gg[DIM][DIM], H[D][DIM];
      element_state<DIM, D>(e, ne, elems, dphi, u, ul, gg, H);
      const double vT = vol[e];
      sp += vT * fd_density<DIM, D, MODEL>(ul, gg, H, lc, j, eps, mp, bad);
      sm += vT * fd_density<DIM, D, MODEL>(ul, gg, H, lc, j, -eps, mp, bad);
    }
    g[t] = (sp - sm) / (2.0 * eps) - b[i * D + j];
  }
  if (bad) atomicOr(status, kStatusDomain);
}

// Expand the stored gradients (l = 1..dim) to the paper's full dphi layout in the caller's
// element order; grad(phi_0) = -sum_{l>=1} grad(phi_l).
template <int DIM>
__global__ void k_expand(int64_t ne, const double* __restrict__ dphi, const double* __restrict__ vol,
                         const int32_t* __restrict__ eperm, double* __restrict__ out,
                         double* __restrict__ vol_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    const int64_t eu = eperm ? (int64_t)eperm[e] : e;
    double* o = out + eu * (DIM + 1) * DIM;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      double s0 = 0.0;
#pragma unroll
      for (int l = 1; l <= DIM; ++l) {
        const double x = dphi[((int64_t)(l - 1) * DIM + m) * ne + e];
        o[l * DIM + m] = x;
        s0 = __dsub_rn(s0, x);
      }
      o[m] = s0;
    }
    vol_out[eu] = vol[e];
  }
}

// ---- dispatch -------------------------------------------------------------------------------

template <int DIM, int D, int MODEL>
fe_status eval_t(fe_ctx* c, const double* v, double* J, double* dens, double* g, bool want_energy,
                 bool want_grad) {
  cudaStream_t s = c->stream;
  const ModelParams mp = model_params(c);
  const int nb_node = grid_for(c->nn, kMaxNodeBlocks);
  const int nb_elem = grid_for(c->ne, kMaxElemBlocks);
  double* node_partials = c->partials + kMaxElemBlocks;
  prof_begin(c, kStagePrep);
  k_node_prep<D, MODEL == FE_NEOHOOKE, DIM><<<nb_node, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b,
                                                                         c->u, node_partials, input_is_disp(c),
                                                                         input_is_disp(c) ? c->bX : 0.0);
  prof_end(c, kStagePrep);
  c->launches++;
  const bool E = want_energy, G = want_grad, Dn = dens != nullptr;
#define FE_ELEM(EN, GR, DE)                                                                         \
  k_elem_f64<DIM, D, MODEL, EN, GR, DE><<<nb_elem, kThreads, 0, s>>>(                               \
      c->ne, c->elems, c->dphi, c->vol, c->u, c->slot, c->eperm, mp, c->r, dens, c->partials,       \
      node_partials, nb_node, c->counter, J, c->status)
  if (c->ne > 0 || E) {
    prof_begin(c, kStageElem);
    if (E && G && Dn) FE_ELEM(true, true, true);
    else if (E && G) FE_ELEM(true, true, false);
    else if (E && Dn) FE_ELEM(true, false, true);
    else if (E) FE_ELEM(true, false, false);
    else if (G && Dn) FE_ELEM(false, true, true);
    else if (G) FE_ELEM(false, true, false);
    else FE_ELEM(false, false, true);
    prof_end(c, kStageElem);
    c->launches++;
  }
#undef FE_ELEM
  if (G) {
    prof_begin(c, kStageGather);
    const fe_status gs = launch_gather_bulk<D, AccF64>(c, c->r, g);
    prof_end(c, kStageGather);
    if (gs) return gs;
    c->launches++;
  }
  return cuda_check(cudaGetLastError(), "eval f64 launch");
}

template <int DIM, int D, int MODEL>
fe_status fd_t(fe_ctx* c, const double* v, double eps, double* g, const int64_t* dofs, int64_t ndofs,
               double* rfd, int32_t* iperm) {
  cudaStream_t s = c->stream;
  const ModelParams mp = model_params(c);
  const int nb_node = grid_for(c->nn, kMaxNodeBlocks);
  prof_begin(c, kStagePrep);
  k_node_prep<D, MODEL == FE_NEOHOOKE, DIM><<<nb_node, kThreads, 0, s>>>(
      c->nn, v, c->X, io_perm(c), c->b, c->u, c->partials + kMaxElemBlocks, input_is_disp(c),
      input_is_disp(c) ? c->bX : 0.0);
  prof_end(c, kStagePrep);
  c->launches++;
  if (dofs) {
    if (ndofs > 0) {
      prof_begin(c, kStageFdGather);
      k_fd_subset<DIM, D, MODEL><<<grid_for(ndofs, 4 * kMaxNodeBlocks), kThreads, 0, s>>>(
          ndofs, dofs, iperm, c->nn, c->ne, c->row_ptr, c->ent, c->elems, c->dphi, c->vol, c->u, c->b,
          c->dir, mp, eps, g, c->status);
      prof_end(c, kStageFdGather);
      c->launches++;
    }
  } else if constexpr (MODEL == FE_NEOHOOKE) {
    if (c->ne > 0) {
      prof_begin(c, kStageFdElem);
      k_elem_fd_nh_f64<DIM><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, s>>>(
          c->ne, c->elems, c->dphi, c->vol, c->u, c->slot, mp, eps, c->r, c->status);
      prof_end(c, kStageFdElem);
      c->launches++;
    }
    prof_begin(c, kStageFdGather);
    const fe_status gs = launch_gather_bulk<D, AccF64>(c, c->r, g);
    prof_end(c, kStageFdGather);
    if (gs) return gs;
    c->launches++;
  } else {
    const int64_t nslot = c->ne * (DIM + 1) * D;
    if (c->ne > 0) {
      prof_begin(c, kStageFdElem);
      k_elem_fd_f64<DIM, D, MODEL><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, s>>>(
          c->ne, c->elems, c->dphi, c->vol, c->u, c->slot, mp, eps, rfd, rfd + nslot, c->status);
      prof_end(c, kStageFdElem);
      c->launches++;
    }
    prof_begin(c, kStageFdGather);
    k_gather_fd<D><<<grid_for(c->nn, 4 * kMaxNodeBlocks), kThreads, 0, s>>>(
        c->nn, c->row_ptr, rfd, rfd + nslot, eps, c->b, c->dir, io_perm(c), g);
    prof_end(c, kStageFdGather);
    c->launches++;
  }
  return cuda_check(cudaGetLastError(), "fd f64 launch");
}

}  // namespace

ModelParams model_params(const fe_ctx* c) {
  ModelParams mp;
  mp.p = c->p;
  mp.C1 = c->C1;
  mp.D1 = c->D1;
  mp.twoC1 = 2.0 * c->C1;
  mp.twoD1 = 2.0 * c->D1;
  mp.pcase = (c->p == 2.0) ? 2 : (c->p == 3.0) ? 3 : 0;
  mp.nn = c->nn;
  return mp;
}

fe_status launch_eval_f64(fe_ctx* c, const double* v, double* J, double* dens, double* g,
                          bool want_energy, bool want_grad) {
  if (c->model == FE_NEOHOOKE) {
    if (c->dim == 2) return eval_t<2, 2, FE_NEOHOOKE>(c, v, J, dens, g, want_energy, want_grad);
    return eval_t<3, 3, FE_NEOHOOKE>(c, v, J, dens, g, want_energy, want_grad);
  }
  if (c->model == FE_PLAPLACE_LP) {
    if (c->dim == 2) return eval_t<2, 1, FE_PLAPLACE_LP>(c, v, J, dens, g, want_energy, want_grad);
    return eval_t<3, 1, FE_PLAPLACE_LP>(c, v, J, dens, g, want_energy, want_grad);
  }
  if (c->dim == 2) return eval_t<2, 1, FE_PLAPLACE>(c, v, J, dens, g, want_energy, want_grad);
  return eval_t<3, 1, FE_PLAPLACE>(c, v, J, dens, g, want_energy, want_grad);
}

// v (caller order) -> u (device order) and the b.v partials, as the first step of an
// FP64 evaluation (used by the Hessian-vector product).
fe_status launch_node_prep_f64(fe_ctx* c, const double* v) {
  const int nb = grid_for(c->nn, kMaxNodeBlocks);
  double* np = c->partials + kMaxElemBlocks;
  const bool disp = input_is_disp(c);
  const double sh = disp ? c->bX : 0.0;
  cudaStream_t s = c->stream;
  if (c->model == FE_NEOHOOKE) {
    if (c->dim == 2) k_node_prep<2, true, 2><<<nb, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b, c->u, np, disp, sh);
    else k_node_prep<3, true, 3><<<nb, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b, c->u, np, disp, sh);
  } else {
    if (c->dim == 2) k_node_prep<1, false, 2><<<nb, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b, c->u, np, false, 0.0);
    else k_node_prep<1, false, 3><<<nb, kThreads, 0, s>>>(c->nn, v, c->X, io_perm(c), c->b, c->u, np, false, 0.0);
  }
  c->launches++;
  return cuda_check(cudaGetLastError(), "node preparation");
}

fe_status launch_fd_f64(fe_ctx* c, const double* v, double eps, double* g, const int64_t* dofs,
                        int64_t ndofs) {
  double* rfd = nullptr;
  int32_t* iperm = nullptr;
  cudaStream_t s = c->stream;
  fe_status st;
  if (!dofs && c->model != FE_NEOHOOKE) {
    const size_t bytes = sizeof(double) * 2 * (size_t)c->ne * (c->dim + 1) * c->d;
    if ((st = cuda_check(cudaMallocAsync((void**)&rfd, bytes > 0 ? bytes : 8, s), "alloc fd"))) return st;
  } else if (io_perm(c)) {
    if ((st = cuda_check(cudaMallocAsync((void**)&iperm, sizeof(int32_t) * c->nn, s), "alloc iperm")))
      return st;
    std::vector<int32_t> ip(c->nn);
    for (int64_t k = 0; k < c->nn; ++k) ip[c->perm_h[k]] = (int32_t)k;
    cudaMemcpyAsync(iperm, ip.data(), sizeof(int32_t) * c->nn, cudaMemcpyHostToDevice, s);
    if ((st = cuda_check(cudaStreamSynchronize(s), "iperm"))) return st;
  }
  if (c->model == FE_NEOHOOKE)
    st = (c->dim == 2) ? fd_t<2, 2, FE_NEOHOOKE>(c, v, eps, g, dofs, ndofs, rfd, iperm)
                       : fd_t<3, 3, FE_NEOHOOKE>(c, v, eps, g, dofs, ndofs, rfd, iperm);
  else if (c->model == FE_PLAPLACE_LP)
    st = (c->dim == 2) ? fd_t<2, 1, FE_PLAPLACE_LP>(c, v, eps, g, dofs, ndofs, rfd, iperm)
                       : fd_t<3, 1, FE_PLAPLACE_LP>(c, v, eps, g, dofs, ndofs, rfd, iperm);
  else
    st = (c->dim == 2) ? fd_t<2, 1, FE_PLAPLACE>(c, v, eps, g, dofs, ndofs, rfd, iperm)
                       : fd_t<3, 1, FE_PLAPLACE>(c, v, eps, g, dofs, ndofs, rfd, iperm);
  if (rfd) cudaFreeAsync(rfd, s);
  if (iperm) cudaFreeAsync(iperm, s);
  return st;
}

fe_status launch_expand_dphi(fe_ctx* c, double* dphi_full, double* vol_user) {
  if (c->ne == 0) return FE_OK;
  if (c->dim == 2)
    k_expand<2><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, c->stream>>>(c->ne, c->dphi, c->vol,
                                                                             c->eperm, dphi_full, vol_user);
  else
    k_expand<3><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, c->stream>>>(c->ne, c->dphi, c->vol,
                                                                             c->eperm, dphi_full, vol_user);
  c->launches++;
  return cuda_check(cudaGetLastError(), "expand launch");
}

}  // namespace fe
