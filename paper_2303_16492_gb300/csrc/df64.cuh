// Double-float ("df64") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two floats (about 48 significant bits).  Built
// from the error-free transformations of Knuth (two-sum, TAOCP vol. 2) and
// Dekker (fast two-sum; two-product, here through a fused multiply-add), with
// one Newton correction for reciprocal and square root.  Used for the scaled
// variant's Gram factorisation and triangular solves, where native FP64 is
// about 60x slower than FP32 on this GPU.
#pragma once

namespace trsgd {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df64{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64{s, b - (s - a)};
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  const df64 t = df_two_sum(a.lo, b.lo);
  const df64 u = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(u.hi, u.lo + t.lo);
}

__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.hi, -a.lo}; }

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// c - a * b with one renormalisation: the leading product a.hi b.hi is split
// exactly (Dekker's two-product through an FMA), its difference with c.hi is
// formed exactly (Knuth's two-sum), and the remaining small terms (the
// product's error, the cross terms, c.lo) are added in float before a final
// fast two-sum.  15 float operations instead of the 27 of df_add(c, -df_mul(a, b)); the extra
// rounding is a float rounding of terms of relative size 2^-24, so the
// result keeps about 44 of the 48 bits.
__device__ __forceinline__ df64 df_fnms_fast(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  const float s = c.hi - p;
  const float bb = s - c.hi;
  const float err = (c.hi - (s - bb)) + (-p - bb);
  float lo = c.lo - e;
  lo = fmaf(-a.hi, b.lo, lo);
  lo = fmaf(-a.lo, b.hi, lo);
  lo += err;
  return df_fast_two_sum(s, lo);
}

// 1 / b: the fast approximate float reciprocal (relative error d0 of a few
// ulp) refined by one Newton-Raphson step r = r0 + r0 (1 - b r0) (the
// double-length reciprocal of Karp and Markstein, "High-precision division
// and square root", ACM TOMS 1997), with the residual 1 - b.hi r0 formed
// exactly by an FMA.  Relative error about d0^2 + 2^-46, i.e. 44 bits; one
// approximate reciprocal instead of two IEEE divisions on the critical path.
__device__ __forceinline__ df64 df_rcp(df64 b) {
  const float r0 = __fdividef(1.f, b.hi);
  const float p = b.hi * r0;
  const float pe = fmaf(b.hi, r0, -p);
  const float e = ((1.f - p) - pe) - b.lo * r0;
  return df_fast_two_sum(r0, r0 * e);
}

__device__ __forceinline__ df64 df_sqrt(df64 a) {
  const float s = sqrtf(a.hi);
  if (!(s > 0.f)) return df64{s, 0.f};
  const df64 r = df_add(a, df_neg(df_mul(df64{s, 0.f}, df64{s, 0.f})));
  return df_fast_two_sum(s, r.hi / (2.f * s));
}

__device__ __forceinline__ df64 df_from_double(double d) {
  const float h = __double2float_rn(d);
  return df64{h, __double2float_rn(d - (double)h)};
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

}  // namespace trsgd
