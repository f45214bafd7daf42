// density_f64.cuh -- the FP64 densities of eqs. neoHook and pLaplacian, shared by the FP64
// element kernels and the no-allocation energy.  Internal linkage: every translation unit
// that includes this header holds its own copy.
#pragma once

#include "fe_internal.cuh"
#include "phi_f64.cuh"  // phi(x) = x - log(1 + x) and 1/(1 + x) from the breakpoint table

namespace fe {
namespace {

// ---- densities --------------------------------------------------------------------------

// Compressible Neo-Hookean density (eq. neoHook) at F = I + H in displacement form:
// delta = det F - 1 = tr H + q with q = i2(H) + det H (3D: q = M00 + H00 X + H01 C01 + H02 C02,
// the row-0 cofactor expansion of det(I + H) minus its O(1) and trace terms), and
//   W = C1 (|H|^2 - 2 q + 2 phi(delta)) + D1 delta^2,
// the same value as C1 (I1 - dim - 2 log det F) + D1 (det F - 1)^2 with rounding relative to
// the size of W instead of C1 dim.  +Inf (and bad) when det F <= 0.
template <int DIM>
__device__ __forceinline__ double nh_density_disp(const double H[DIM][DIM], const ModelParams& mp, bool& bad) {
  double tr = 0.0, hsq = 0.0, q;
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    tr += H[j][j];
#pragma unroll
    for (int m = 0; m < DIM; ++m) hsq = fma(H[j][m], H[j][m], hsq);
  }
  if constexpr (DIM == 3) {
    const double M00 = H[1][1] * H[2][2] - H[1][2] * H[2][1];
    const double X = H[1][1] + H[2][2] + M00;
    const double C01 = H[1][2] * H[2][0] - H[1][0] * (1.0 + H[2][2]);
    const double C02 = H[1][0] * H[2][1] - (1.0 + H[1][1]) * H[2][0];
    q = M00 + H[0][0] * X + H[0][1] * C01 + H[0][2] * C02;
  } else {
    q = H[0][0] * H[1][1] - H[0][1] * H[1][0];
  }
  const double delta = tr + q;
  if (!(1.0 + delta > 0.0)) {
    bad = true;
    return CUDART_INF;
  }
  return mp.C1 * (hsq - 2.0 * q + 2.0 * phi_f64(delta)) + mp.D1 * delta * delta;
}

__device__ __forceinline__ double plap_density(double s, const ModelParams& mp) {
  if (mp.pcase == 2) return 0.5 * s;
  if (mp.pcase == 3) return s * sqrt(s) * (1.0 / 3.0);
  return s > 0.0 ? pow(s, 0.5 * mp.p) / mp.p : 0.0;
}

// Componentwise p-Laplacian (FE_PLAPLACE_LP): |a|^p and |a|^(p-2) of one gradient component.
__device__ __forceinline__ void plap_lp_terms(double a, const ModelParams& mp, double* ap, double* ap2) {
  const double x = fabs(a);
  if (mp.pcase == 2) {
    *ap = x * x;
    *ap2 = 1.0;
  } else if (mp.pcase == 3) {
    *ap = x * x * x;
    *ap2 = x;
  } else if (x > 0.0) {
    *ap2 = pow(x, mp.p - 2.0);
    *ap = *ap2 * x * x;
  } else {
    *ap = *ap2 = 0.0;
  }
}

__device__ __forceinline__ double plap_coef(double s, const ModelParams& mp) {
  if (mp.pcase == 2) return 1.0;
  if (mp.pcase == 3) return sqrt(s);
  return s > 0.0 ? pow(s, 0.5 * (mp.p - 2.0)) : 0.0;
}

}  // namespace
}  // namespace fe
