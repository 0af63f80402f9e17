// lst_ff.cuh -- float-float ("double-single") arithmetic on FP32 operations: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant
// bits. Used by the FP32 T5-DNN score path (features and network), whose result must stay
// within 1e-6 of an FP64 evaluation although the trained networks amplify a single FP32
// rounding of an input or a hidden activation beyond that.
//
// Methods: error-free sum (Knuth, TAOCP vol. 2, Section 4.2.2, "two-sum") and product
// through a fused multiply-add (the residual a*b - fl(a*b) is a float); Dekker's
// double-length operations (Numer. Math. 18, 1971) for add, multiply, divide and square
// root; the compensated dot product Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput.
// 26, 2005). The logarithm reduces x = m 2^e with m in [1/sqrt 2, sqrt 2) and sums the
// series ln m = 2 (s + s^3/3 + s^5/5 + ...) with s = (m - 1)/(m + 1), |s| < 0.172: the
// leading term in float-float, the rest (below 2e-3) in FP32, so the absolute error stays
// near 1e-10. The library is built with -fmad=false, so no a*b+c below is contracted
// unless written as an FMA, which the error-free forms rely on.
#pragma once
#include "lst_internal.cuh"

namespace lstk {

__device__ __forceinline__ ff ff_make(float a) { return {a, 0.0f}; }
// a + b = s + e exactly
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// a + b = s + e exactly, given |a| >= |b| or a == 0
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
// a * b = p + e exactly (barring underflow)
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = a * b;
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  const ff t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  p.lo += x.hi * y.lo + x.lo * y.hi;
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mulf(ff x, float b) {
  ff p = two_prod(x.hi, b);
  p.lo = __fmaf_rn(x.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
// x / y: three quotient digits, each from the remainder of the previous ones
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  const float q1 = x.hi / y.hi;
  ff r = ff_sub(x, ff_mulf(y, q1));
  const float q2 = r.hi / y.hi;
  r = ff_sub(r, ff_mulf(y, q2));
  const float q3 = r.hi / y.hi;
  return ff_add(quick_two_sum(q1, q2), ff_make(q3));
}
__device__ __forceinline__ ff ff_divf(ff x, float b) { return ff_div(x, ff_make(b)); }
// sqrt(x), x >= 0: one Newton correction of the FP32 root
__device__ __forceinline__ ff ff_sqrt(ff x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float y = sqrtf(x.hi);
  const ff yy = two_prod(y, y);
  const float r = (((x.hi - yy.hi) - yy.lo) + x.lo) / (2.0f * y);
  return quick_two_sum(y, r);
}
// u.x^2 + u.y^2 of a float-float vector
__device__ __forceinline__ ff ff_norm2(ff ux, ff uy) { return ff_add(ff_mul(ux, ux), ff_mul(uy, uy)); }

// ln 2 and 1 / ln 10 split into a float and the float nearest to the remainder
constexpr float LN2_HI = 0.6931472f, LN2_LO = -1.9046542e-09f;
constexpr float INV_LN10_HI = 0.4342945f, INV_LN10_LO = -1.010305e-08f;

// natural logarithm of x > 0 (a normal float-float)
__device__ __forceinline__ ff ff_log(ff x) {
  const unsigned bits = __float_as_uint(x.hi);
  int e = (int)((bits >> 23) & 0xffu) - 127;
  float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);    // [1, 2)
  if (m > 1.41421356f) {
    m *= 0.5f;
    e += 1;
  }
  const float scale = __uint_as_float((unsigned)(127 - e) << 23);     // 2^-e, exact
  const ff mm = {m, x.lo * scale};
  const ff s = ff_div(ff_add(mm, ff_make(-1.0f)), ff_add(mm, ff_make(1.0f)));
  const float s2 = s.hi * s.hi;
  float p = 1.0f / 17.0f;
  p = 1.0f / 15.0f + s2 * p;
  p = 1.0f / 13.0f + s2 * p;
  p = 1.0f / 11.0f + s2 * p;
  p = 1.0f / 9.0f + s2 * p;
  p = 1.0f / 7.0f + s2 * p;
  p = 1.0f / 5.0f + s2 * p;
  p = 1.0f / 3.0f + s2 * p;
  const ff half_ln_m = ff_add(s, ff_make((s.hi * s2) * p));
  const ff ln_m = {2.0f * half_ln_m.hi, 2.0f * half_ln_m.lo};
  const ff ln2 = {LN2_HI, LN2_LO};
  return ff_add(ff_mulf(ln2, (float)e), ln_m);
}
__device__ __forceinline__ ff ff_log10(ff x) { return ff_mul(ff_log(x), ff{INV_LN10_HI, INV_LN10_LO}); }
// asinh(v) = sign(v) ln(|v| + sqrt(v^2 + 1))
__device__ __forceinline__ ff ff_asinh(ff v) {
  const bool neg = v.hi < 0.0f;
  const ff a = neg ? ff_neg(v) : v;
  const ff r = ff_log(ff_add(a, ff_sqrt(ff_add(ff_mul(a, a), ff_make(1.0f)))));
  return neg ? ff_neg(r) : r;
}
__device__ __forceinline__ ff ff_abs(ff x) { return x.hi < 0.0f ? ff_neg(x) : x; }
// x < y for normalised float-float values
__device__ __forceinline__ bool ff_lt(ff x, ff y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

}  // namespace lstk
