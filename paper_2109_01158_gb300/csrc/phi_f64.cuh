// phi_f64.cuh -- phi(x) = x - log(1 + x) and 1/(1 + x) in FP64 from a breakpoint table,
// shared by the FP64 element kernels.  The table and the functions have internal linkage:
// every translation unit that includes this header holds its own copy.
#pragma once

#include "fe_internal.cuh"

namespace fe {
namespace {

// ---- phi(x) = x - log(1 + x), x > -1 --------------------------------------------------------
//
// Breakpoints c_j = (j - FE_PHI_J0) / 1024 with F_j = 1 + c_j (the table covers
// [-306/1024, 306/1024]; the kernels use it for |x| < 306/1024 = 76.5/256): the nearest
// breakpoint gives x = c_j + f with |f| <= 1/2048 (exact: c_j is a multiple of 2^-10 within
// a factor 2 of x, Sterbenz' lemma), and with r = f / F_j
//   phi(x) = (c_j - ln F_j) + f (1 - 1/F_j) + (r - log1p(r)),
//   r - log1p(r) = r^2 (1/2 - r/3 + r^2/4 - r^3/5 + r^4/6) + O(r^7),
// |r| < 7.0e-4, so the truncation is below 2^-54 of r - log1p(r).  The three terms never
// cancel by more than about a factor 4, the table holds c_j - ln F_j to twice double
// precision (hi + lo), and there is no division.  Outside: x - log1p(x).
#include "phi_table_f64.h"

struct __align__(32) PhiRow {
  double a_hi, a_lo, b, r;   // c_j - ln F_j (hi + lo), 1 - 1/F_j, 1/F_j
};
__device__ const PhiRow kPhiTab[FE_PHI_N] = {FE_PHI_TABLE_ROWS};

__device__ __noinline__ double phi_f64_wide(double x) { return x - log1p(x); }

// |x| < 76.5/256 by the bit pattern (an integer compare; NaN fails it): the symmetric part of
// the table interval, the rest of it goes to log1p
__device__ __forceinline__ bool in_phi_table(double x) {
  constexpr long long kAbs = 0x3FD3200000000000LL;   // bits of 76.5/256 = 0.298828125
  return (__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL) < kAbs;
}

// Row j of the table, f = x - c_j (exact) and r = f / F_j for x inside it.
struct PhiArg {
  double2 A, BR;
  double f, r;
};

__device__ __forceinline__ PhiArg phi_arg(double x) {
  // round(FE_PHI_SCALE x) by the 1.5 * 2^52 shift: t = 1.5 * 2^52 + round(FE_PHI_SCALE x) exactly
  const double t = fma(x, (double)FE_PHI_SCALE, 0x1.8p52);
  int j = __double2loint(t) + FE_PHI_J0;
  j = min(max(j, 0), FE_PHI_N - 1);
  const double2* row = reinterpret_cast<const double2*>(kPhiTab + j);
  PhiArg a;
  a.A = __ldg(row);
  a.BR = __ldg(row + 1);
  a.f = fma(t - 0x1.8p52, -1.0 / FE_PHI_SCALE, x);   // x - c_j, exact (product and sum)
  a.r = a.f * a.BR.y;
  return a;
}

__device__ __forceinline__ double phi_from(const PhiArg& a) {
  const double r = a.r;
  double p = 1.0 / 6.0;
  p = fma(p, r, -1.0 / 5.0);
  p = fma(p, r, 1.0 / 4.0);
  p = fma(p, r, -1.0 / 3.0);
  p = fma(p, r, 1.0 / 2.0);
  const double psi = (r * r) * p;
  return a.A.x + (a.A.y + fma(a.f, a.BR.x, psi));
}

__device__ __forceinline__ double phi_f64(double x) {
  if (!in_phi_table(x)) return phi_f64_wide(x);
  return phi_from(phi_arg(x));
}

// 1/(1 + x) from the same row: inside the table 1 + x = F_j (1 + r), so
// 1/(1 + x) = (1/F_j)(1 - r + r^2 - ... - r^5) (|r| < 7.0e-4: the next term is below
// 2^-62 of the sum), which replaces a division.
__device__ __forceinline__ double rcp_from(const PhiArg& a) {
  const double r = a.r;
  double s = 1.0 - r;
#pragma unroll
  for (int k = 0; k < 4; ++k) s = fma(-r, s, 1.0);
  return a.BR.y * s;
}

__device__ __forceinline__ double rcp1p_f64(double x) {
  if (!in_phi_table(x)) return 1.0 / (1.0 + x);
  return rcp_from(phi_arg(x));
}

// phi(x) and 1/(1 + x) together (the reciprocal bitwise equal to rcp1p_f64's).
__device__ __forceinline__ double phi_rcp_f64(double x, double* rcp) {
  if (!in_phi_table(x)) {
    *rcp = 1.0 / (1.0 + x);
    return phi_f64_wide(x);
  }
  const PhiArg a = phi_arg(x);
  *rcp = rcp_from(a);
  return phi_from(a);
}

}  // namespace
}  // namespace fe
