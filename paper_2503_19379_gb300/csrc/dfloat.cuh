// Double-float ("float-float") arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits. Built from the error-free transformations
//   two_sum(a, b):  s = fl(a + b), e = (a - (s - bb)) + (b - bb), bb = s - a   (Knuth), a + b = s + e exactly;
//   two_prod(a, b): p = fl(a b),   e = fma(a, b, -p),                             a b = p + e exactly;
// (Dekker 1971; Hida, Li and Bailey, "Library for double-double and quad-double arithmetic", 2001).
// On GB300 the FP32 pipe is ~62x faster than the FP64 pipe, so the FP64-accurate parts of the mixed-precision solve
// (the block X, its operator image, the X-X Gram block) run in this format: ~10 FP32 operations per operation, a
// relative error of ~2^-44 instead of 2^-53, which the eigensolver does not resolve (its FP64 residual floor is
// ~1e-10 here).
#pragma once
#include <cuda_runtime.h>

namespace pc {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ double df_to(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  df r;
  r.hi = a + b;
  r.lo = b - (r.hi - a);
  return r;
}
__device__ __forceinline__ df two_sum(float a, float b) {
  df r;
  r.hi = a + b;
  const float bb = r.hi - a;
  r.lo = (a - (r.hi - bb)) + (b - bb);
  return r;
}
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return quick_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}
// multiplication by a power of two (exact)
__device__ __forceinline__ df df_scale2(df x, float s) { return df{x.hi * s, x.lo * s}; }

// complex double-float
struct cdf {
  df re, im;
};
__device__ __forceinline__ cdf cdf_from(double2 z) { return cdf{df_from(z.x), df_from(z.y)}; }
__device__ __forceinline__ double2 cdf_to(cdf z) { return make_double2(df_to(z.re), df_to(z.im)); }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
  return cdf{df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ cdf cdf_mulc(cdf a, cdf b) {
  return cdf{df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return cdf{df_mul(a.re, s), df_mul(a.im, s)}; }

// s += a b for double-float a, b, s: the product's rounding error is exact via fma, the sum via two_sum, then one
// renormalisation (15 FP32 operations); about 2^-44 relative per step
__device__ __forceinline__ void df_mac(df &s, df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s = quick_two_sum(t, err + (s.lo + e));
}
// s += a b for complex double-float
__device__ __forceinline__ void cdf_mac(cdf &s, cdf a, cdf b) {
  df_mac(s.re, a.re, b.re);
  df_mac(s.re, df_neg(a.im), b.im);
  df_mac(s.im, a.re, b.im);
  df_mac(s.im, a.im, b.re);
}
__device__ __forceinline__ cdf cdf_scale2(cdf a, float s) { return cdf{df_scale2(a.re, s), df_scale2(a.im, s)}; }

// A double-float sum built term by term without renormalising after every term: s is the FP32 running sum of the
// leading products, e collects every rounding error exactly captured on the way (two_sum of the running sum, the
// fma residual of each leading product) plus the small cross terms hi*lo + lo*hi. One term costs 12 FP32 operations
// (df_mac: 15), and the value is quick_two_sum(s, e) at the end; e stays ~2^-24 |s|, so its own rounding is ~2^-48
// of the sum, like the renormalised form.
struct dfsum {
  float s, e;
};
// a += x c
__device__ __forceinline__ void dfsum_mac(dfsum &a, df x, df c) {
  const float p = x.hi * c.hi;
  const float ep = fmaf(x.hi, c.hi, -p);
  const float t = a.s + p;
  const float bb = t - a.s;
  const float es = (a.s - (t - bb)) + (p - bb);
  a.s = t;
  a.e += es + ep;
  a.e = fmaf(x.hi, c.lo, a.e);
  a.e = fmaf(x.lo, c.hi, a.e);
}
// a += f for an FP32 f
__device__ __forceinline__ void dfsum_addf(dfsum &a, float f) {
  const float t = a.s + f;
  const float bb = t - a.s;
  a.e += (a.s - (t - bb)) + (f - bb);
  a.s = t;
}
__device__ __forceinline__ df dfsum_value(dfsum a) { return quick_two_sum(a.s, a.e); }
// x + f for a double-float x and an FP32 f
__device__ __forceinline__ df df_addf(df x, float f) {
  const df s = two_sum(x.hi, f);
  return quick_two_sum(s.hi, s.lo + x.lo);
}

// Storage of complex double-float blocks. The solver keeps its FP64-accurate block as pairs (re.hi, re.lo, im.hi,
// im.lo) in one float4 (16 bytes, like complex128), so that its kernels read and write it without conversions:
// converting a double to a pair costs four FP64-pipe instructions and back three, more FP64 work than the
// double-float arithmetic does in FP32. complex128 blocks (the public entry points) convert on load and store.
__device__ __forceinline__ cdf ld_cdf(const double2 *p) { return cdf_from(*p); }
__device__ __forceinline__ cdf ld_cdf(const float4 *p) {
  const float4 v = *p;
  return cdf{df{v.x, v.y}, df{v.z, v.w}};
}
__device__ __forceinline__ void st_cdf(double2 *p, cdf z) { *p = cdf_to(z); }
__device__ __forceinline__ void st_cdf(float4 *p, cdf z) { *p = make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo); }
// FP64 value of a stored element (for the FP64 checks and conversions off the iteration path)
__device__ __forceinline__ double2 ld_c128(const double2 *p) { return *p; }
__device__ __forceinline__ double2 ld_c128(const float2 *p) {
  const float2 v = *p;
  return make_double2((double)v.x, (double)v.y);
}
__device__ __forceinline__ double2 ld_c128(const float4 *p) {
  const float4 v = *p;
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

}  // namespace pc
