// elem_f32.cuh -- the per-element work of the FP32 path (not in the paper; its precision
// variant): H = grad u, W(F) and |T| dW/dF of eq. neoHook / eq. pLaplacian in float.
//
// Written in displacement form so that no O(1) quantities cancel: with F = I + H
// (H = grad u, u = v - X),
//   delta = det F - 1 = tr H + i2(H) + det H      (i2: sum of principal 2x2 minors; 2D: tr H + det H)
//   I1 - dim - 2 log det F = |H|^2 - 2 (i2(H) + det H) + 2 phi(delta),   phi(x) = x - log(1+x)
//   dW/dF = 2 C1 (F - F^{-T}) + 2 D1 delta cof F,   F - F^{-T} = H + cof(F) H^T / det F
// phi uses the series of 2 atanh: with s = x/(2+x), log(1+x) = 2(s + s^3/3 + s^5/5 + ...),
// so phi(x) = s x - 2 s^3 (1/3 + s^2/5 + s^4/7 + ...).  Where |delta| > 1/2 (det F far from
// 1, or close to 0), delta, log det F and 1/det F are taken in FP64.
#pragma once

#include "df64.cuh"
#include "fe_internal.cuh"

namespace fe {
namespace {

// phi(x) = x - log(1+x) for |x| <= 1/2 by the atanh series (|s| <= 1/3, 8 terms).
__device__ __forceinline__ float phi_series_f32(float x) {
  const float s = __fdividef(x, __fadd_rn(2.0f, x));
  const float s2 = __fmul_rn(s, s);
  float t = 1.0f / 17.0f;
  t = fmaf(t, s2, 1.0f / 15.0f);
  t = fmaf(t, s2, 1.0f / 13.0f);
  t = fmaf(t, s2, 1.0f / 11.0f);
  t = fmaf(t, s2, 1.0f / 9.0f);
  t = fmaf(t, s2, 1.0f / 7.0f);
  t = fmaf(t, s2, 1.0f / 5.0f);
  t = fmaf(t, s2, 1.0f / 3.0f);
  return fmaf(s, x, __fmul_rn(__fmul_rn(-2.0f, s), __fmul_rn(s2, t)));
}

// 1/x for x in [1/2, 3/2] (here x = det F near 1): the hardware's approximate reciprocal
// (rcp.approx, one instruction) refined by one Newton step r (2 - x r), written as
// r + r (1 - x r) with FMAs; within about an ulp of the float reciprocal, which is all the
// gradient's FP32 arithmetic needs, at a third of the instructions of the correctly rounded one.
__device__ __forceinline__ float rcp_newton(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.f), r);
}

// a b - c d with one rounding of the second product (the same contraction in every kernel)
__device__ __forceinline__ float det2f(float a, float b, float c, float d) { return fmaf(a, b, -__fmul_rn(c, d)); }

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

// u_l - u_0 to float accuracy from double-float nodal values: the hi difference is exact when
// the two values are within a factor 2 (Sterbenz' lemma), otherwise within half an ulp of a
// result of the same size; adding the (tiny) lo difference and rounding once leaves at most
// about one float ulp of the difference.  (Rounding u itself to float first would lose the
// factor by which u exceeds its differences across an element.)
// The two differences are one paired instruction (b * -1 + a: a - b rounded once).
__device__ __forceinline__ float pair_diff(float2 a, float2 b) {
  const float2 d = __ffma2_rn(b, make_float2(-1.f, -1.f), a);
  return __fadd_rn(d.x, d.y);
}

// One element in float: from the differences a[l][j] = (u_{l+1} - u_0)_j (l = 0..DIM-1) and
// the stored gradients g[l][m] = d phi_{l+1} / dx_m, forms H_jm = sum_l a[l][j] g[l][m] (eq. Dv),
// returns W (when WANT_W; +Inf and bad = true when det F <= 0) and, when GRAD, P = |T| dW/dF.
template <int DIM, int D, int MODEL, bool WANT_W, bool GRAD>
__device__ __forceinline__ float elem_f32(const float (&a)[DIM][D], const float (&g)[DIM][DIM], float vT,
                                          float C1, float D1, const ModelParams& mp, float (&P)[D][DIM],
                                          bool& bad) {
  // every product and sum is an explicit fmaf or _rn intrinsic (or its paired form, two
  // independent operations in one instruction, rounded the same way): the compiler cannot
  // contract them differently in the energy-only and the gradient instantiations, which
  // therefore give bitwise the same W (and the two gradient instantiations the same P)
  float H[D][DIM];
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      float s = __fmul_rn(a[0][j], g[0][m]);
#pragma unroll
      for (int l = 1; l < DIM; ++l) s = fmaf(a[l][j], g[l][m], s);
      H[j][m] = s;
    }
  float W = 0.f;
  if constexpr (MODEL == FE_NEOHOOKE) {
    // |H|^2 with two accumulators (the even and the odd row-major entries, one paired
    // instruction per two entries), added at the end
    float hsq;
    {
      const float* Hf = &H[0][0];
      float2 acc = __fmul2_rn(make_float2(Hf[0], Hf[1]), make_float2(Hf[0], Hf[1]));
#pragma unroll
      for (int f = 2; f + 1 < DIM * DIM; f += 2)
        acc = __ffma2_rn(make_float2(Hf[f], Hf[f + 1]), make_float2(Hf[f], Hf[f + 1]), acc);
      hsq = __fadd_rn(acc.x, acc.y);
      if (DIM * DIM % 2) hsq = fmaf(Hf[DIM * DIM - 1], Hf[DIM * DIM - 1], hsq);
    }
    float tr, q, C[DIM][DIM];  // q = i2(H) + det H, C = cof(I + H)
    if constexpr (DIM == 3) {
      tr = __fadd_rn(__fadd_rn(H[0][0], H[1][1]), H[2][2]);
      const float m00 = det2f(H[1][1], H[2][2], H[1][2], H[2][1]);
      const float m01 = det2f(H[1][2], H[2][0], H[1][0], H[2][2]);
      const float m02 = det2f(H[1][0], H[2][1], H[1][1], H[2][0]);
      const float m11 = det2f(H[0][0], H[2][2], H[0][2], H[2][0]);
      const float m22 = det2f(H[0][0], H[1][1], H[0][1], H[1][0]);
      const float dH = fmaf(H[0][0], m00, fmaf(H[0][1], m01, __fmul_rn(H[0][2], m02)));
      q = __fadd_rn(__fadd_rn(__fadd_rn(m00, m11), m22), dH);
      if (GRAD) {
        const float F00 = __fadd_rn(1.f, H[0][0]), F11 = __fadd_rn(1.f, H[1][1]), F22 = __fadd_rn(1.f, H[2][2]);
        C[0][0] = det2f(F11, F22, H[1][2], H[2][1]);
        C[0][1] = det2f(H[1][2], H[2][0], H[1][0], F22);
        C[0][2] = det2f(H[1][0], H[2][1], F11, H[2][0]);
        C[1][0] = det2f(H[0][2], H[2][1], H[0][1], F22);
        C[1][1] = det2f(F00, F22, H[0][2], H[2][0]);
        C[1][2] = det2f(H[0][1], H[2][0], F00, H[2][1]);
        C[2][0] = det2f(H[0][1], H[1][2], H[0][2], F11);
        C[2][1] = det2f(H[0][2], H[1][0], F00, H[1][2]);
        C[2][2] = det2f(F00, F11, H[0][1], H[1][0]);
      }
    } else {
      tr = __fadd_rn(H[0][0], H[1][1]);
      q = det2f(H[0][0], H[1][1], H[0][1], H[1][0]);
      if (GRAD) {
        C[0][0] = __fadd_rn(1.f, H[1][1]);
        C[0][1] = -H[1][0];
        C[1][0] = -H[0][1];
        C[1][1] = __fadd_rn(1.f, H[0][0]);
      }
    }
    float delta = __fadd_rn(tr, q);
    bool ebad = false;
    float phi2 = 0.f;     // 2 phi(delta)
    float inv_det = 1.f;  // 1 / det F
    const bool far = !(fabsf(delta) <= 0.5f);
    if (!far) {
      if (WANT_W) phi2 = __fmul_rn(2.f, phi_series_f32(delta));
      if (GRAD) inv_det = rcp_newton(__fadd_rn(1.f, delta));
    }
    // Far from F = I: det F and log det F in FP64, in a called function behind a warp vote
    // so that the compiler cannot if-convert it into every element's path.
    if (__any_sync(__activemask(), far) && far) {
      float Hf[9];
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) Hf[j * DIM + m] = H[j][m];
      ebad = !far_from_identity_f64(Hf, DIM, &delta, &phi2, &inv_det);
    }
    // W = C1 (|H|^2 - 2 q + 2 phi(delta)) + D1 delta^2
    if (WANT_W) W = fmaf(C1, __fadd_rn(fmaf(-2.f, q, hsq), phi2), __fmul_rn(D1, __fmul_rn(delta, delta)));
    if (ebad) {
      W = CUDART_INF_F;
      bad = true;
    }
    if (GRAD) {
      // P = 2 C1 (H + C H^T / det F) + 2 D1 delta C, scaled by |T|
      const float aa = __fmul_rn(__fmul_rn(2.f, C1), vT);
      const float c = __fmul_rn(__fmul_rn(__fmul_rn(2.f, D1), delta), vT);
      const float ai = __fmul_rn(aa, inv_det);
      float ch[DIM][DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          float t = __fmul_rn(C[j][0], H[m][0]);  // (C H^T)_jm = sum_k C_jk H_mk
#pragma unroll
          for (int k = 1; k < DIM; ++k) t = fmaf(C[j][k], H[m][k], t);
          ch[j][m] = t;
        }
      // P elementwise, two entries per paired instruction (row-major order)
      const float* Hf = &H[0][0];
      const float* Cf = &C[0][0];
      const float* chf = &ch[0][0];
      float* Pf = &P[0][0];
      const float2 aa2 = make_float2(aa, aa), ai2 = make_float2(ai, ai), c2 = make_float2(c, c);
#pragma unroll
      for (int f = 0; f + 1 < DIM * DIM; f += 2) {
        const float2 t = __ffma2_rn(aa2, make_float2(Hf[f], Hf[f + 1]),
                                    __ffma2_rn(ai2, make_float2(chf[f], chf[f + 1]),
                                               __fmul2_rn(c2, make_float2(Cf[f], Cf[f + 1]))));
        Pf[f] = t.x;
        Pf[f + 1] = t.y;
      }
      if (DIM * DIM % 2) {
        const int f = DIM * DIM - 1;
        Pf[f] = fmaf(aa, Hf[f], fmaf(ai, chf[f], __fmul_rn(c, Cf[f])));
      }
    }
  } else {
    float s = __fmul_rn(H[0][0], H[0][0]);
#pragma unroll
    for (int m = 1; m < DIM; ++m) s = fmaf(H[0][m], H[0][m], s);
    if (WANT_W) {
      if (mp.pcase == 2) W = __fmul_rn(0.5f, s);
      else if (mp.pcase == 3) W = __fmul_rn(__fmul_rn(s, sqrtf(s)), 1.f / 3.f);
      else W = s > 0.f ? __fdiv_rn(powf(s, 0.5f * (float)mp.p), (float)mp.p) : 0.f;
    }
    if (GRAD) {
      float cf = (mp.pcase == 2) ? 1.f : (mp.pcase == 3) ? sqrtf(s)
                                   : (s > 0.f ? powf(s, 0.5f * (float)(mp.p - 2.0)) : 0.f);
      cf = __fmul_rn(cf, vT);
#pragma unroll
      for (int m = 0; m < DIM; ++m) P[0][m] = __fmul_rn(cf, H[0][m]);
    }
  }
  return W;
}

}  // namespace
}  // namespace fe
