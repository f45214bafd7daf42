// elem_df.cuh -- per-element and per-node work of the double-float (FE_DF64) path, shared
// by the single-mesh kernels (fe_eval_df64.cu) and the batched kernels (fe_batch.cu) so that
// both compute bit-identical element values.
#pragma once

#include "df64.cuh"
#include "fe_internal.cuh"

namespace fe {

__device__ __forceinline__ df ld_df(const float2* __restrict__ p, int64_t i) {
  const float2 a = __ldg(p + i);
  return {a.x, a.y};
}

// Loads of data that other blocks of the same launch write (the persistent batched kernel):
// ordinary cached loads (ld.global.ca), never the read-only path (ld.global.nc), which is
// not kept coherent with writes made during the launch.  The caller has synchronised with
// the writers first (an acquire at GPU scope, then a block barrier), after which ordinary
// loads see the written values, and neighbouring elements still share the L1 lines of
// their nodes.
template <bool COH, class T>
__device__ __forceinline__ T ld_ro(const T* p) {
  if constexpr (COH) return __ldca(p);
  else return __ldg(p);
}

// Node record of the double-float displacement: D pairs, padded to 4 pairs in 3D.
template <int D, bool COH = false>
__device__ __forceinline__ void load_u_df(const float2* __restrict__ u, int32_t n, df* out) {
  if (D == 1) {
    const float2 a = ld_ro<COH>(u + n);
    out[0] = {a.x, a.y};
  } else if (D == 2) {
    const float4 a = ld_ro<COH>(reinterpret_cast<const float4*>(u) + n);
    out[0] = {a.x, a.y};
    out[1] = {a.z, a.w};
  } else {
    const float4* p = reinterpret_cast<const float4*>(u) + 2 * (int64_t)n;
    const float4 a = ld_ro<COH>(p), b = ld_ro<COH>(p + 1);
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
static __device__ __noinline__ void plap_general_f64(double s, double p, double* W, double* coef) {
  *W = s > 0.0 ? pow(s, 0.5 * p) / p : 0.0;
  *coef = s > 0.0 ? pow(s, 0.5 * (p - 2.0)) : 0.0;
}

// phi(x) = x - log(1 + x) for x > -1.  For |x| <= 1/16 by the series of 2 atanh without any
// cancellation: with s = x / (2 + x), phi = s x - 2 s^3 (1/3 + s^2/5 + s^4/7 + s^6/9 + s^8/11)
// (|s| < 1/31, truncation below 2^-50 relative); otherwise x - log(1 + x) with the
// table-driven logarithm (the difference then keeps about 2^-40 of phi).
__device__ __forceinline__ df df_phi(df x, const LogEntry* tab) {
  if (fabsf(x.hi) <= 0.0625f) {
    const df s = df_mul(x, df_rcp(df_add_f(x, 2.0f)));
    const df s2 = df_sqr(s);
    const float t1 = fmaf(s2.hi, 1.0f / 11.0f, 1.0f / 9.0f);
    df t = df_add(df{0x1.24924ap-3f, -0x1.b6db6ep-28f}, df_mul_f(s2, t1));         // 1/7 + s^2 t1
    t = df_fma(s2, t, df{0x1.99999ap-3f, -0x1.99999ap-29f});                      // 1/5 + s^2 t
    t = df_fma(s2, t, df{0x1.555556p-2f, -0x1.555556p-27f});                      // 1/3 + s^2 t
    const df s3 = df_mul(s2, s);
    return df_sub(df_mul(s, x), df_scale(df_mul(s3, t), 2.0f));
  }
  return df_sub(x, df_log(df_add_f(x, 1.0f), tab));
}

template <int DIM>
struct MatDF {
  df m[DIM][DIM];
};

// |T| dW/dF near F = I without O(1) terms: 2 C1 (H - L) + 2 delta (D1 + C1 / det F) cof F with
// L = cof F - I, whose diagonal L_jj is formed from H (X0 = L_00 from the caller).  Out of
// line: the common path keeps the registers and code of the plain form.
template <int DIM>
static __device__ __noinline__ MatDF<DIM> nh_stress_small_df(MatDF<DIM> H, MatDF<DIM> C, df X0, df delta, df rJ,
                                                             df a, df vT, df C1, df D1) {
  df Ld[DIM];
  if constexpr (DIM == 3) {
    Ld[0] = X0;
    Ld[1] = df_add(df_add(H.m[0][0], H.m[2][2]), df_det2(H.m[0][0], H.m[2][2], H.m[0][2], H.m[2][0]));
    Ld[2] = df_add(df_add(H.m[0][0], H.m[1][1]), df_det2(H.m[0][0], H.m[1][1], H.m[0][1], H.m[1][0]));
  } else {
    Ld[0] = H.m[1][1];
    Ld[1] = H.m[0][0];
  }
  const df cp = df_mul(vT, df_scale(df_mul(delta, df_add(D1, df_mul(C1, rJ))), 2.f));
  MatDF<DIM> P;
#pragma unroll
  for (int j = 0; j < DIM; ++j)
#pragma unroll
    for (int m = 0; m < DIM; ++m) P.m[j][m] = df_dot2(a, df_sub(H.m[j][m], j == m ? Ld[j] : C.m[j][m]), cp, C.m[j][m]);
  return P;
}

// One element: gathers the nodal values, forms H = grad u (eq. Dv) and returns W(F) when
// WANT_W (eq. neoHook or eq. pLaplacian); when GRAD, also writes the local forces
// r_{T,l} = |T| dW/dF grad(phi_l) (Sec. 6.2) to the CSR slots.  vT receives |T|; `bad` is set
// when det F <= 0.  Arrays are the structure-of-arrays of fe_ctx with stride ne.  COH: the
// nodal values u were written earlier in the same launch (coherent loads).
template <int DIM, int D, int MODEL, bool WANT_W, bool GRAD, bool COH = false>
__device__ __forceinline__ df elem_df_one(int64_t e, int64_t ne, const int32_t* __restrict__ elems,
                                          const float2* __restrict__ dphi, const float2* __restrict__ vol,
                                          const float2* __restrict__ u, const int32_t* __restrict__ slot,
                                          const ModelDF& md, const LogEntry* tab, float2* __restrict__ r,
                                          bool& bad, df& vT) {
  constexpr int K = DIM + 1;
    df ul[K][D];
#pragma unroll
    for (int l = 0; l < K; ++l) load_u_df<D, COH>(u, __ldg(elems + (int64_t)l * ne + e), ul[l]);
    df g[DIM][DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l)
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[l][m] = ld_df(dphi, ((int64_t)l * DIM + m) * ne + e);
    vT = ld_df(vol, e);
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
      // Displacement form of eq. neoHook with F = I + H (the same value, no cancellation of
      // O(1) terms):  delta = det F - 1 = tr H + q with q = i2(H) + det H, and
      //   I1 - dim - 2 log det F = |H|^2 - 2 q + 2 phi(delta),   phi(x) = x - log(1 + x).
      df F[DIM][DIM], C[DIM][DIM];
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int m = 0; m < DIM; ++m) F[j][m] = (j == m) ? df_add_f(H[j][m], 1.0f) : H[j][m];
      df tr = H[0][0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) tr = df_add(tr, H[j][j]);
      df q, X0 = {0.f, 0.f};
      if (DIM == 3) {
        // C00 = 1 + X with X = H11 + H22 + M00 (M00 the minor of H); then
        // q = M00 + H00 X + H01 C01 + H02 C02 exactly in real arithmetic
        const df M00 = df_det2(H[1][1], H[DIM - 1][DIM - 1], H[1][DIM - 1], H[DIM - 1][1]);
        const df X = df_add(df_add(H[1][1], H[DIM - 1][DIM - 1]), M00);
        X0 = X;
        C[0][0] = df_add_f(X, 1.0f);
        C[0][1] = df_det2(F[1][2], F[2][0], F[1][0], F[2][2]);
        C[0][2] = df_det2(F[1][0], F[2][1], F[1][1], F[2][0]);
        q = df_add(M00, df_dot3(H[0][0], X, H[0][1], C[0][1], H[0][DIM - 1], C[0][DIM - 1]));
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
        q = df_det2(H[0][0], H[1][1], H[0][1], H[1][0]);   // det H
      }
      const df delta = df_add(tr, q);
      const df det = df_add_f(delta, 1.0f);
      const bool ebad = !(det.hi > 0.f);
      if (WANT_W) {
        const df hsq = df_sumsq<D * DIM>(&H[0][0]);
        const df phi = ebad ? df{0.f, 0.f} : df_phi(delta, tab);
        const df br = df_add(df_add(hsq, df_scale(q, -2.f)), df_scale(phi, 2.f));
        W = df_dot2(md.C1, br, md.D1, df_sqr(delta));
        if (ebad) W = {CUDART_INF_F, 0.f};
      }
      if (GRAD) {
        // dW/dF = 2 C1 F + (2 D1 (det F - 1) - 2 C1 / det F) cof F, times |T|.  Near F = I the
        // two terms cancel to O(|H|); a warp with any |H|^2 < 1e-4 uses the same value as
        //   2 C1 (H - L) + 2 delta (D1 + C1 / det F) cof F,   L = cof F - I,
        // with the diagonal L_jj formed from H without the 1 (no O(1) term left).
        const df rJ = df_rcp(det);
        const df a = df_mul(md.twoC1, vT);
        float hs = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int m = 0; m < DIM; ++m) hs = fmaf(H[j][m].hi, H[j][m].hi, hs);
        if (__any_sync(__activemask(), hs < 1e-4f)) {
          MatDF<DIM> h, cf;
#pragma unroll
          for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int m = 0; m < DIM; ++m) {
              h.m[j][m] = H[j][m];
              cf.m[j][m] = C[j][m];
            }
          const MatDF<DIM> p = nh_stress_small_df<DIM>(h, cf, X0, delta, rJ, a, vT, md.C1, md.D1);
#pragma unroll
          for (int j = 0; j < DIM; ++j)
#pragma unroll
            for (int m = 0; m < DIM; ++m) P[j][m] = p.m[j][m];
        } else {
          const df c = df_mul(vT, df_dot2(md.twoD1, delta, md.negTwoC1, rJ));
#pragma unroll
          for (int j = 0; j < D; ++j)
#pragma unroll
            for (int m = 0; m < DIM; ++m) P[j][m] = df_dot2(a, F[j][m], c, C[j][m]);
        }
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
    if (GRAD) {
      df r0[D];
#pragma unroll
      for (int l = 1; l <= DIM; ++l) {
        const int64_t q = __ldg(slot + (int64_t)l * ne + e);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const df s = (DIM == 3) ? df_dot3(P[j][0], g[l - 1][0], P[j][1], g[l - 1][1], P[j][DIM - 1], g[l - 1][DIM - 1])
                                  : df_dot2(P[j][0], g[l - 1][0], P[j][DIM - 1], g[l - 1][DIM - 1]);
          r[q * D + j] = make_float2(s.hi, s.lo);
          r0[j] = (l == 1) ? df_neg(s) : df_sub(r0[j], s);   // (the first term needs no addition)
        }
      }
      const int64_t q0 = __ldg(slot + e);
#pragma unroll
      for (int j = 0; j < D; ++j) r[q0 * D + j] = make_float2(r0[j].hi, r0[j].lo);
    }
    return W;
}

}  // namespace fe
