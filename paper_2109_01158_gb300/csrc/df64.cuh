// df64.cuh -- double-float arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, which carries
// about 48 significand bits.  GB300 executes 128 FP32 FMAs per SM per clock but only 2 FP64
// FMAs, so a few FP32 operations per double-float operation are far cheaper than one FP64
// operation.
//
// Building blocks (error-free transformations):
//   TwoSum (Knuth, TAOCP vol. 2): s + e = a + b exactly, 6 flops.
//   FastTwoSum (Dekker 1971): s + e = a + b exactly when |a| >= |b| (or a = 0), 3 flops.
//   TwoProd with FMA: p + e = a * b exactly, 2 flops.
// Double-word operations follow Joldes, Muller & Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic" (ACM TOMS 44(2), 2017): the "sloppy"
// sum (absolute error of order u^2 (|x| + |y|), u = 2^-24), the DW x DW and DW x FP products
// with FMA (relative error below 5u^2), and one Newton step for the reciprocal and the
// square root.  The logarithm is table driven (Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990): argument
// reduction by a power of two and a table point, then the Taylor series of log(1+t).
//
// Range: as for float, |values| must stay within about 1e-30 .. 1e30 for the low word to
// keep its precision (ample for FEM energies in SI or scaled units).
#pragma once

#include <cuda_runtime.h>

namespace fe {

struct df {
  float hi, lo;
};

// Every addition and multiplication inside the error-free transformations below is written
// with the _rn intrinsics: nvcc would otherwise fuse a product into a following sum (FMA
// contraction), which breaks the exactness of TwoSum / FastTwoSum and makes the result
// depend on how the compiler schedules each kernel.
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ df df_from(float a) { return {a, 0.f}; }

// Round a double to the nearest double-float (hi = fl(x), lo = fl(x - hi)).
__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(__dsub_rn(x, (double)h))};
}

__device__ __forceinline__ double df_to_double(df x) { return __dadd_rn((double)x.hi, (double)x.lo); }

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = fadd(a, b);
  const float bp = fsub(s, a);
  const float e = fadd(fsub(a, fsub(s, bp)), fsub(b, bp));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = fadd(a, b);
  return {s, fsub(b, fsub(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = fmul(a, b);
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

// x + y, "sloppy" double-word sum (11 flops).
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(x.lo, y.lo)));
}

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x + b for a float b (10 flops).
__device__ __forceinline__ df df_add_f(df x, float b) {
  const df s = two_sum(x.hi, b);
  return fast_two_sum(s.hi, fadd(s.lo, x.lo));
}

// x * y (DW x DW with FMA, 7 flops).
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = fmul(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// x * b for a float b (5 flops).
__device__ __forceinline__ df df_mul_f(df x, float b) {
  const float p = fmul(x.hi, b);
  float e = fmaf(x.hi, b, -p);
  e = fmaf(x.lo, b, e);
  return fast_two_sum(p, e);
}

// x * 2^k is exact: scale both words.
__device__ __forceinline__ df df_scale(df x, float pow2) { return {fmul(x.hi, pow2), fmul(x.lo, pow2)}; }

__device__ __forceinline__ df df_sqr(df x) {
  const float p = fmul(x.hi, x.hi);
  float e = fmaf(x.hi, x.hi, -p);
  e = fmaf(fmul(2.f, x.hi), x.lo, e);
  return fast_two_sum(p, e);
}

// x * y + z (the product's leading part is exact; 15 flops).
__device__ __forceinline__ df df_fma(df x, df y, df z) {
  const float p = fmul(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  const df s = two_sum(p, z.hi);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(e, z.lo)));
}

// a*b + c*d with both leading products exact and one TwoSum (about 19 flops).
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
  const float p = fmul(a.hi, b.hi), q = fmul(c.hi, d.hi);
  float e = fmaf(a.hi, b.hi, -p);
  float f = fmaf(c.hi, d.hi, -q);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  f = fmaf(c.hi, d.lo, f);
  f = fmaf(c.lo, d.hi, f);
  const df s = two_sum(p, q);
  return fast_two_sum(s.hi, fadd(s.lo, fadd(e, f)));
}

// a*b - c*d
__device__ __forceinline__ df df_det2(df a, df b, df c, df d) { return df_dot2(a, b, df_neg(c), d); }

// a0*b0 + a1*b1 + a2*b2 (leading products exact, two TwoSums; about 31 flops).
__device__ __forceinline__ df df_dot3(df a0, df b0, df a1, df b1, df a2, df b2) {
  const float p0 = fmul(a0.hi, b0.hi), p1 = fmul(a1.hi, b1.hi), p2 = fmul(a2.hi, b2.hi);
  float e0 = fmaf(a0.hi, b0.hi, -p0);
  float e1 = fmaf(a1.hi, b1.hi, -p1);
  float e2 = fmaf(a2.hi, b2.hi, -p2);
  e0 = fmaf(a0.hi, b0.lo, e0);
  e0 = fmaf(a0.lo, b0.hi, e0);
  e1 = fmaf(a1.hi, b1.lo, e1);
  e1 = fmaf(a1.lo, b1.hi, e1);
  e2 = fmaf(a2.hi, b2.lo, e2);
  e2 = fmaf(a2.lo, b2.hi, e2);
  const df s = two_sum(p0, p1);
  const df t = two_sum(s.hi, p2);
  return fast_two_sum(t.hi, fadd(fadd(t.lo, s.lo), fadd(e0, fadd(e1, e2))));
}

// 1/x by one Newton step from the float reciprocal (about 12 flops).
__device__ __forceinline__ df df_rcp(df x) {
  const float r = __frcp_rn(x.hi);
  const df p = df_mul_f(x, r);                    // ~ 1
  const float e = fsub(fsub(1.0f, p.hi), p.lo);   // 1 - p.hi is exact (Sterbenz)
  return fast_two_sum(r, fmul(r, e));
}

// sqrt(x) for x >= 0 by one Newton step from the float square root.
__device__ __forceinline__ df df_sqrt(df x) {
  if (!(x.hi > 0.f)) return {0.f, 0.f};
  const float y = __fsqrt_rn(x.hi);
  const df yy = two_prod(y, y);
  const float r = fadd(fsub(fsub(x.hi, yy.hi), yy.lo), x.lo);   // x - y^2 to float precision
  return fast_two_sum(y, fmul(r, __fdiv_rn(0.5f, y)));
}

// ---- natural logarithm ---------------------------------------------------------------------

// Table of the logarithm: for i = 0..kLogTable-1, the point c_i = kLogC0 + i / 256 covers
// [sqrt(1/2), sqrt(2)]; entry i holds r_i = float(1 / c_i) and L_i = -log(r_i) as a double-float.
constexpr int kLogTable = 184;
constexpr float kLogC0 = 0.703125f;

struct LogEntry {
  float r, Lhi, Llo, pad;
};

// log(x) for x > 0.  Absolute error about 2^-48 |log x| + 2^-52.
__device__ __forceinline__ df df_log(df x, const LogEntry* tab) {
  // x = 2^k m with m in [sqrt(1/2), sqrt(2))
  const int bits = __float_as_int(x.hi);
  int k = ((bits >> 23) & 0xff) - 127;
  float mh = __int_as_float((bits & 0x007fffff) | 0x3f800000);   // in [1, 2)
  if (mh > 1.41421356f) {
    mh *= 0.5f;
    k += 1;
  }
  const float scale = __int_as_float((127 - k) << 23);            // 2^-k, exact
  const df m = df_scale(x, scale);
  // table point and t = m r - 1 (|t| <= about 2^-8.5)
  int i = __float2int_rn((m.hi - kLogC0) * 256.0f);
  i = i < 0 ? 0 : (i > kLogTable - 1 ? kLogTable - 1 : i);
  const LogEntry T = tab[i];
  // t = m r - 1 formed exactly up to the last, tiny term: both partial products are exact
  // (TwoProd) and pa.hi - 1 is exact (Sterbenz), so t keeps its full relative precision
  // even though m r is close to 1.
  const df pa = two_prod(m.hi, T.r);
  const df pb = two_prod(m.lo, T.r);
  df t = two_sum(fsub(pa.hi, 1.0f), pa.lo);
  t = df_add_f(t, pb.hi);
  t = df_add_f(t, pb.lo);
  // log(1 + t) = t - t^2/2 + t^3/3 - t^4/4 + t^5/5 - t^6/6 + ...
  const df t2 = df_sqr(t);
  const df t3 = df_mul(t2, t);
  const df third = df_mul(t3, df{0x1.555556p-2f, -0x1.555556p-27f});   // 1/3 as a double-float
  const float th = t.hi;
  const float rest = t3.hi * (th * (-0.25f + th * (0.2f + th * (-0.166666672f + th * 0.142857149f))));
  df l1p = df_add(t, df_scale(t2, -0.5f));
  l1p = df_add(l1p, third);
  l1p = df_add_f(l1p, rest);
  // k log 2 + L_i + log(1 + t); log 2 as a double-float
  const df kln2 = df_mul_f(df{0x1.62e430p-1f, -0x1.05c610p-29f}, (float)k);
  return df_add(df_add(kln2, df{T.Lhi, T.Llo}), l1p);
}

}  // namespace fe
