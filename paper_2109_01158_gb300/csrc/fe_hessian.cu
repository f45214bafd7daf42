// fe_hessian.cu -- Hessian-vector products of the discrete energy (FP64):
//   Hw = d/dt grad J(v + t w) at t = 0 on the free dofs,
// the second derivative of J_grad = sum |T| W(F_T) (Sec. 1) along w, gathered over the nodal
// patches like the exact gradient (Sec. 6.2); b.v has no second derivative.  Entries of w on
// Dirichlet dofs are taken as 0 and Dirichlet rows of Hw are 0.
//
// Pipeline (context stream):
//   k_node_prep   v -> u (the same kernel as the gradient)
//   k_w_prep      w (caller order) -> device order, Dirichlet entries zeroed
//   k_hvp_f64     one thread per element: H and dF = sum_{l>=1} (w_l - w_0) grad(phi_l)^T,
//                 the directional derivative dP of dW/dF along dF, local contributions
//                 |T| dP grad(phi_l) to the CSR slots
//   k_gather_bulk per-node patch sums (no load term)
// Neo-Hookean: with cof = cof F and d(cof) its derivative along dF,
//   dP = 2 C1 dF + (2 C1 / det^2 + 2 D1) (cof : dF) cof + (2 D1 (det - 1) - 2 C1 / det) d(cof);
// every term is O(|dF|), so no O(1) terms cancel near F = I.  p-Laplacian, s = |grad v|^2:
//   dP = s^((p-2)/2) dF + (p - 2) s^((p-4)/2) (grad v . dF) grad v,  dP = dF for p = 2 and
//   0 at grad v = 0 otherwise; componentwise p-Laplacian: dP_m = (p - 1) |v_m|^(p-2) dF_m.
#include "fe_internal.cuh"
#include "gather_bulk.cuh"

namespace fe {
namespace {

template <int D>
__device__ __forceinline__ void load_vec(const double* __restrict__ u, int32_t n, double* out) {
  if (D == 1) {
    out[0] = __ldg(u + n);
  } else if (D == 2) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(u) + n);
    out[0] = a.x;
    out[1] = a.y;
  } else {
    const double2* p = reinterpret_cast<const double2*>(u) + 2 * (int64_t)n;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    out[0] = a.x;
    out[1] = a.y;
    out[2] = b.x;
  }
}

// w (caller dof order) -> device order in the padded node layout of u, 0 on Dirichlet dofs.
template <int D>
__global__ void __launch_bounds__(kThreads) k_w_prep(int64_t nn, const double* __restrict__ w,
                                                     const int32_t* __restrict__ perm,
                                                     const uint8_t* __restrict__ dir, double* __restrict__ wd,
                                                     const int* skip) {
  constexpr int DP = D == 3 ? 4 : D;
  if (skip && *skip) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
    const int64_t src = perm ? (int64_t)perm[i] : i;
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      double x = 0.0;
      if (j < D && !dir[i * D + j]) x = w[src * D + j];
      wd[i * DP + j] = x;
    }
  }
}

template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_hvp_f64(int64_t ne, const int32_t* __restrict__ elems,
                                                      const double* __restrict__ dphi, const double* __restrict__ vol,
                                                      const double* __restrict__ u, const double* __restrict__ wd,
                                                      const int32_t* __restrict__ slot, ModelParams mp,
                                                      double* __restrict__ r, int* status, const int* skip) {
  constexpr int K = DIM + 1;
  if (skip && *skip) return;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    double ul[K][D], wl[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) {
      const int32_t n = __ldg(elems + (int64_t)l * ne + e);
      load_vec<D>(u, n, ul[l]);
      load_vec<D>(wd, n, wl[l]);
    }
    double g[DIM][DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = __ldg(dphi + ((int64_t)l * DIM + m) * ne + e);
    const double vT = __ldg(vol + e);
    double H[D][DIM], dF[D][DIM];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double a[DIM], b[DIM];
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        a[l] = ul[l + 1][j] - ul[0][j];
        b[l] = wl[l + 1][j] - wl[0][j];
      }
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        double s = a[0] * g[0][m], t = b[0] * g[0][m];
#pragma unroll
        for (int l = 1; l < DIM; ++l) {
          s = fma(a[l], g[l][m], s);
          t = fma(b[l], g[l][m], t);
        }
        H[j][m] = s;
        dF[j][m] = t;
      }
    }
    double dP[D][DIM];
    if constexpr (MODEL == FE_NEOHOOKE) {
      double F[DIM][DIM], C[DIM][DIM], dC[DIM][DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) F[j][m] = (j == m) ? 1.0 + H[j][m] : H[j][m];
      double delta;
      if constexpr (DIM == 3) {
        // cofactors and their derivatives along dF: signed 2x2 minors of the other rows/columns
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const int r0 = j == 0 ? 1 : 0, r1 = j == 2 ? 1 : 2;
            const int c0 = m == 0 ? 1 : 0, c1 = m == 2 ? 1 : 2;
            const double mn = F[r0][c0] * F[r1][c1] - F[r0][c1] * F[r1][c0];
            const double dmn = dF[r0][c0] * F[r1][c1] + F[r0][c0] * dF[r1][c1] - dF[r0][c1] * F[r1][c0] -
                               F[r0][c1] * dF[r1][c0];
            const double sg = ((j + m) & 1) ? -1.0 : 1.0;
            C[j][m] = sg * mn;
            dC[j][m] = sg * dmn;
          }
        // det F - 1 without the O(1) cancellation: tr H + i2(H) + det H via the row-0 expansion
        const double M00 = H[1][1] * H[2][2] - H[1][2] * H[2][1];
        const double X = H[1][1] + H[2][2] + M00;
        delta = H[0][0] + X + H[0][0] * X + H[0][1] * C[0][1] + H[0][2] * C[0][2];
      } else {
        C[0][0] = F[1][1];
        C[0][1] = -F[1][0];
        C[1][0] = -F[0][1];
        C[1][1] = F[0][0];
        dC[0][0] = dF[1][1];
        dC[0][1] = -dF[1][0];
        dC[1][0] = -dF[0][1];
        dC[1][1] = dF[0][0];
        delta = H[0][0] + H[1][1] + (H[0][0] * H[1][1] - H[0][1] * H[1][0]);
      }
      const double det = 1.0 + delta;
      if (!(det > 0.0)) bad = true;
      double cdf = 0.0;
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) cdf = fma(C[j][m], dF[j][m], cdf);
      const double rdet = 1.0 / det;
      const double a = 2.0 * mp.C1 * vT;
      const double bcoef = vT * (2.0 * mp.C1 * rdet * rdet + 2.0 * mp.D1) * cdf;
      const double ccoef = vT * (2.0 * mp.D1 * delta - 2.0 * mp.C1 * rdet);
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) dP[j][m] = fma(a, dF[j][m], fma(bcoef, C[j][m], ccoef * dC[j][m]));
    } else if constexpr (MODEL == FE_PLAPLACE_LP) {
      // dP_m = (p - 1) |H_m|^(p-2) dF_m (dF_m for p = 2)
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        const double x = fabs(H[0][m]);
        double c;
        if (mp.pcase == 2) c = 1.0;
        else if (mp.pcase == 3) c = 2.0 * x;
        else c = (x > 0.0) ? (mp.p - 1.0) * pow(x, mp.p - 2.0) : 0.0;
        dP[0][m] = vT * c * dF[0][m];
      }
    } else {
      double s = 0.0, hd = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        s = fma(H[0][m], H[0][m], s);
        hd = fma(H[0][m], dF[0][m], hd);
      }
      double c1, c2;
      if (mp.pcase == 2) {
        c1 = 1.0;
        c2 = 0.0;
      } else if (s > 0.0) {
        c1 = (mp.pcase == 3) ? sqrt(s) : pow(s, 0.5 * (mp.p - 2.0));
        c2 = (mp.p - 2.0) * c1 / s;
      } else {
        c1 = c2 = 0.0;
      }
#pragma unroll
      for (int m = 0; m < DIM; ++m) dP[0][m] = vT * fma(c1, dF[0][m], c2 * hd * H[0][m]);
    }
    // local contributions dP grad(phi_l) (l >= 1); l = 0 gets minus their sum
    double r0[D];
#pragma unroll
    for (int l = 1; l <= DIM; ++l) {
      const int64_t q = __ldg(slot + (int64_t)l * ne + e);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        double s = dP[j][0] * g[l - 1][0];
#pragma unroll
        for (int m = 1; m < DIM; ++m) s = fma(dP[j][m], g[l - 1][m], s);
        r[q * D + j] = s;
        r0[j] = (l == 1) ? -s : r0[j] - s;
      }
    }
    const int64_t q0 = __ldg(slot + e);
#pragma unroll
    for (int j = 0; j < D; ++j) r[q0 * D + j] = r0[j];
  }
  if (bad) atomicOr(status, kStatusDomain);
}

// ---- products at a fixed point (the inner CG of a Newton step) ---------------------------
//
// Within one CG solve v is fixed, so the part of k_hvp_f64 that depends on v alone is computed
// once (k_hvp_prep_f64) into a structure-of-arrays cache, and each product (k_hvp_cached_f64)
// reads it instead of gathering u and rebuilding F, cof F and the coefficients.  Both kernels
// evaluate the same expressions as k_hvp_f64.  Cache entries per element:
//   Neo-Hookean            F, cof F, 2 C1 |T|, |T| (2 C1 / det^2 + 2 D1), |T| (2 D1 (det - 1) - 2 C1 / det)
//   componentwise p-Lap.   |T| (p - 1) |H_m|^(p-2)                       (m < dim)
//   p-Laplacian            H, c1 = s^((p-2)/2), c2 = (p - 2) c1 / s, |T|

template <int DIM, int MODEL>
constexpr int hvp_cache_width() {
  return MODEL == FE_NEOHOOKE ? 2 * DIM * DIM + 3 : (MODEL == FE_PLAPLACE_LP ? DIM : DIM + 3);
}

template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_hvp_prep_f64(int64_t ne, const int32_t* __restrict__ elems,
                                                           const double* __restrict__ dphi,
                                                           const double* __restrict__ vol,
                                                           const double* __restrict__ u, ModelParams mp,
                                                           double* __restrict__ cache, int* status) {
  constexpr int K = DIM + 1;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    double ul[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) load_vec<D>(u, __ldg(elems + (int64_t)l * ne + e), ul[l]);
    double g[DIM][DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = __ldg(dphi + ((int64_t)l * DIM + m) * ne + e);
    const double vT = __ldg(vol + e);
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
    double* out = cache + e;
    if constexpr (MODEL == FE_NEOHOOKE) {
      double F[DIM][DIM], C[DIM][DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) F[j][m] = (j == m) ? 1.0 + H[j][m] : H[j][m];
      double delta;
      if constexpr (DIM == 3) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const int r0 = j == 0 ? 1 : 0, r1 = j == 2 ? 1 : 2;
            const int c0 = m == 0 ? 1 : 0, c1 = m == 2 ? 1 : 2;
            const double mn = F[r0][c0] * F[r1][c1] - F[r0][c1] * F[r1][c0];
            const double sg = ((j + m) & 1) ? -1.0 : 1.0;
            C[j][m] = sg * mn;
          }
        const double M00 = H[1][1] * H[2][2] - H[1][2] * H[2][1];
        const double X = H[1][1] + H[2][2] + M00;
        delta = H[0][0] + X + H[0][0] * X + H[0][1] * C[0][1] + H[0][2] * C[0][2];
      } else {
        C[0][0] = F[1][1];
        C[0][1] = -F[1][0];
        C[1][0] = -F[0][1];
        C[1][1] = F[0][0];
        delta = H[0][0] + H[1][1] + (H[0][0] * H[1][1] - H[0][1] * H[1][0]);
      }
      const double det = 1.0 + delta;
      if (!(det > 0.0)) bad = true;
      const double rdet = 1.0 / det;
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          out[(int64_t)(j * DIM + m) * ne] = F[j][m];
          out[(int64_t)(DIM * DIM + j * DIM + m) * ne] = C[j][m];
        }
      out[(int64_t)(2 * DIM * DIM) * ne] = 2.0 * mp.C1 * vT;
      out[(int64_t)(2 * DIM * DIM + 1) * ne] = vT * (2.0 * mp.C1 * rdet * rdet + 2.0 * mp.D1);
      out[(int64_t)(2 * DIM * DIM + 2) * ne] = vT * (2.0 * mp.D1 * delta - 2.0 * mp.C1 * rdet);
    } else if constexpr (MODEL == FE_PLAPLACE_LP) {
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        const double x = fabs(H[0][m]);
        double c;
        if (mp.pcase == 2) c = 1.0;
        else if (mp.pcase == 3) c = 2.0 * x;
        else c = (x > 0.0) ? (mp.p - 1.0) * pow(x, mp.p - 2.0) : 0.0;
        out[(int64_t)m * ne] = vT * c;
      }
    } else {
      double s = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) s = fma(H[0][m], H[0][m], s);
      double c1, c2;
      if (mp.pcase == 2) {
        c1 = 1.0;
        c2 = 0.0;
      } else if (s > 0.0) {
        c1 = (mp.pcase == 3) ? sqrt(s) : pow(s, 0.5 * (mp.p - 2.0));
        c2 = (mp.p - 2.0) * c1 / s;
      } else {
        c1 = c2 = 0.0;
      }
#pragma unroll
      for (int m = 0; m < DIM; ++m) out[(int64_t)m * ne] = H[0][m];
      out[(int64_t)DIM * ne] = c1;
      out[(int64_t)(DIM + 1) * ne] = c2;
      out[(int64_t)(DIM + 2) * ne] = vT;
    }
  }
  if (bad) atomicOr(status, kStatusDomain);
}

template <int DIM, int D, int MODEL>
__global__ void __launch_bounds__(kThreads) k_hvp_cached_f64(int64_t ne, const int32_t* __restrict__ elems,
                                                             const double* __restrict__ dphi,
                                                             const double* __restrict__ cache,
                                                             const double* __restrict__ wd,
                                                             const int32_t* __restrict__ slot,
                                                             double* __restrict__ r, const int* skip) {
  constexpr int K = DIM + 1;
  if (skip && *skip) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
    double wl[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) load_vec<D>(wd, __ldg(elems + (int64_t)l * ne + e), wl[l]);
    double g[DIM][DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = __ldg(dphi + ((int64_t)l * DIM + m) * ne + e);
    double dF[D][DIM];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double b[DIM];
#pragma unroll
      for (int l = 0; l < DIM; ++l) b[l] = wl[l + 1][j] - wl[0][j];
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        double t = b[0] * g[0][m];
#pragma unroll
        for (int l = 1; l < DIM; ++l) t = fma(b[l], g[l][m], t);
        dF[j][m] = t;
      }
    }
    const double* in = cache + e;
    double dP[D][DIM];
    if constexpr (MODEL == FE_NEOHOOKE) {
      double F[DIM][DIM], C[DIM][DIM], dC[DIM][DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          F[j][m] = __ldg(in + (int64_t)(j * DIM + m) * ne);
          C[j][m] = __ldg(in + (int64_t)(DIM * DIM + j * DIM + m) * ne);
        }
      if constexpr (DIM == 3) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const int r0 = j == 0 ? 1 : 0, r1 = j == 2 ? 1 : 2;
            const int c0 = m == 0 ? 1 : 0, c1 = m == 2 ? 1 : 2;
            const double dmn = dF[r0][c0] * F[r1][c1] + F[r0][c0] * dF[r1][c1] - dF[r0][c1] * F[r1][c0] -
                               F[r0][c1] * dF[r1][c0];
            const double sg = ((j + m) & 1) ? -1.0 : 1.0;
            dC[j][m] = sg * dmn;
          }
      } else {
        dC[0][0] = dF[1][1];
        dC[0][1] = -dF[1][0];
        dC[1][0] = -dF[0][1];
        dC[1][1] = dF[0][0];
      }
      double cdf = 0.0;
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) cdf = fma(C[j][m], dF[j][m], cdf);
      const double a = __ldg(in + (int64_t)(2 * DIM * DIM) * ne);
      const double bcoef = __ldg(in + (int64_t)(2 * DIM * DIM + 1) * ne) * cdf;
      const double ccoef = __ldg(in + (int64_t)(2 * DIM * DIM + 2) * ne);
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) dP[j][m] = fma(a, dF[j][m], fma(bcoef, C[j][m], ccoef * dC[j][m]));
    } else if constexpr (MODEL == FE_PLAPLACE_LP) {
#pragma unroll
      for (int m = 0; m < DIM; ++m) dP[0][m] = __ldg(in + (int64_t)m * ne) * dF[0][m];
    } else {
      double H[DIM], hd = 0.0;
#pragma unroll
      for (int m = 0; m < DIM; ++m) {
        H[m] = __ldg(in + (int64_t)m * ne);
        hd = fma(H[m], dF[0][m], hd);
      }
      const double c1 = __ldg(in + (int64_t)DIM * ne), c2 = __ldg(in + (int64_t)(DIM + 1) * ne);
      const double vT = __ldg(in + (int64_t)(DIM + 2) * ne);
#pragma unroll
      for (int m = 0; m < DIM; ++m) dP[0][m] = vT * fma(c1, dF[0][m], c2 * hd * H[m]);
    }
    double r0[D];
#pragma unroll
    for (int l = 1; l <= DIM; ++l) {
      const int64_t q = __ldg(slot + (int64_t)l * ne + e);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        double s = dP[j][0] * g[l - 1][0];
#pragma unroll
        for (int m = 1; m < DIM; ++m) s = fma(dP[j][m], g[l - 1][m], s);
        r[q * D + j] = s;
        r0[j] = (l == 1) ? -s : r0[j] - s;
      }
    }
    const int64_t q0 = __ldg(slot + e);
#pragma unroll
    for (int j = 0; j < D; ++j) r[q0 * D + j] = r0[j];
  }
}

template <int DIM, int D, int MODEL>
fe_status hvp_prepare_t(fe_ctx* c, const double* v) {
  fe_status st = launch_node_prep_f64(c, v);
  if (st) return st;
  if (c->ne > 0) {
    k_hvp_prep_f64<DIM, D, MODEL><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, c->stream>>>(
        c->ne, c->elems, c->dphi, c->vol, c->u, model_params(c), c->hvp_cache, c->status);
    c->launches++;
  }
  return cuda_check(cudaGetLastError(), "hessian-vector preparation");
}

template <int DIM, int D, int MODEL>
fe_status hvp_cached_t(fe_ctx* c, const double* w, double* Hw, const int* skip) {
  cudaStream_t s = c->stream;
  k_w_prep<D><<<grid_for(c->nn, kMaxNodeBlocks), kThreads, 0, s>>>(c->nn, w, io_perm(c), c->dir, c->w_hvp, skip);
  c->launches++;
  if (c->ne > 0) {
    k_hvp_cached_f64<DIM, D, MODEL><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, s>>>(
        c->ne, c->elems, c->dphi, c->hvp_cache, c->w_hvp, c->slot, c->r, skip);
    c->launches++;
  }
  fe_status st = launch_gather_bulk<D, AccF64>(c, c->r, Hw, nullptr, skip);
  if (st) return st;
  c->launches++;
  return cuda_check(cudaGetLastError(), "cached hessian-vector launch");
}

template <int DIM, int D, int MODEL>
fe_status hvp_dir_t(fe_ctx* c, const double* w, double* Hw, const int* skip) {
  cudaStream_t s = c->stream;
  const ModelParams mp = model_params(c);
  const int nb_node = grid_for(c->nn, kMaxNodeBlocks);
  k_w_prep<D><<<nb_node, kThreads, 0, s>>>(c->nn, w, io_perm(c), c->dir, c->w_hvp, skip);
  c->launches++;
  if (c->ne > 0) {
    k_hvp_f64<DIM, D, MODEL><<<grid_for(c->ne, kMaxElemBlocks), kThreads, 0, s>>>(
        c->ne, c->elems, c->dphi, c->vol, c->u, c->w_hvp, c->slot, mp, c->r, c->status, skip);
    c->launches++;
  }
  fe_status st = launch_gather_bulk<D, AccF64>(c, c->r, Hw, nullptr, skip);
  if (st) return st;
  c->launches++;
  return cuda_check(cudaGetLastError(), "hessian-vector launch");
}

}  // namespace

fe_status launch_hvp_dir_f64(fe_ctx* c, const double* w, double* Hw, const int* skip) {
  if (c->model == FE_NEOHOOKE)
    return c->dim == 2 ? hvp_dir_t<2, 2, FE_NEOHOOKE>(c, w, Hw, skip) : hvp_dir_t<3, 3, FE_NEOHOOKE>(c, w, Hw, skip);
  if (c->model == FE_PLAPLACE_LP)
    return c->dim == 2 ? hvp_dir_t<2, 1, FE_PLAPLACE_LP>(c, w, Hw, skip) : hvp_dir_t<3, 1, FE_PLAPLACE_LP>(c, w, Hw, skip);
  return c->dim == 2 ? hvp_dir_t<2, 1, FE_PLAPLACE>(c, w, Hw, skip) : hvp_dir_t<3, 1, FE_PLAPLACE>(c, w, Hw, skip);
}

// Sized by the components per node (not the model, which a scalar mesh may switch between
// the two p-Laplacians): the widest cache of the models the mesh admits.
size_t hvp_cache_doubles(const fe_ctx* c) {
  const int dim = c->dim;
  const int width = c->d > 1 ? 2 * dim * dim + 3 : dim + 3;
  return (size_t)width * (size_t)c->ne;
}

fe_status launch_hvp_prepare_f64(fe_ctx* c, const double* v) {
  if (c->model == FE_NEOHOOKE)
    return c->dim == 2 ? hvp_prepare_t<2, 2, FE_NEOHOOKE>(c, v) : hvp_prepare_t<3, 3, FE_NEOHOOKE>(c, v);
  if (c->model == FE_PLAPLACE_LP)
    return c->dim == 2 ? hvp_prepare_t<2, 1, FE_PLAPLACE_LP>(c, v) : hvp_prepare_t<3, 1, FE_PLAPLACE_LP>(c, v);
  return c->dim == 2 ? hvp_prepare_t<2, 1, FE_PLAPLACE>(c, v) : hvp_prepare_t<3, 1, FE_PLAPLACE>(c, v);
}

fe_status launch_hvp_cached_f64(fe_ctx* c, const double* w, double* Hw, const int* skip) {
  if (c->model == FE_NEOHOOKE)
    return c->dim == 2 ? hvp_cached_t<2, 2, FE_NEOHOOKE>(c, w, Hw, skip)
                       : hvp_cached_t<3, 3, FE_NEOHOOKE>(c, w, Hw, skip);
  if (c->model == FE_PLAPLACE_LP)
    return c->dim == 2 ? hvp_cached_t<2, 1, FE_PLAPLACE_LP>(c, w, Hw, skip)
                       : hvp_cached_t<3, 1, FE_PLAPLACE_LP>(c, w, Hw, skip);
  return c->dim == 2 ? hvp_cached_t<2, 1, FE_PLAPLACE>(c, w, Hw, skip) : hvp_cached_t<3, 1, FE_PLAPLACE>(c, w, Hw, skip);
}

fe_status launch_hvp_f64(fe_ctx* c, const double* v, const double* w, double* Hw) {
  fe_status st = launch_node_prep_f64(c, v);
  if (st) return st;
  return launch_hvp_dir_f64(c, w, Hw, nullptr);
}

}  // namespace fe
