// ff.cuh -- double-float arithmetic: a value is hi + lo with two floats.
//
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
// FastTwoSum (Dekker, "A floating-point technique for extending the available
// precision", Numer. Math. 18, 1971); TwoProduct through a fused multiply-add.
// A normalised pair carries about 2 * 24 significant bits, which is what the
// stationarity polish needs on GB300, whose FP64 rate is a small fraction of
// its FP32 rate.  The inverse square root is one Newton step on the FP32
// estimate carried out in this arithmetic (relative error ~ the square of the
// estimate's).
#pragma once

namespace fpt {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff{-y.hi, -y.lo}); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  ff p = two_prod(x.hi, y.hi);
  float lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, lo);
}

// x * y for a double-float x and a float y
__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  ff p = two_prod(x.hi, y);
  return fast_two_sum(p.hi, __fmaf_rn(x.lo, y, p.lo));
}

// 1 / sqrt(x) for x > 0: r0 = rsqrtf(x.hi), r = r0 + r0 (1 - x r0^2) / 2
__device__ __forceinline__ ff ff_rsqrt(ff x) {
  const float r0 = rsqrtf(x.hi);
  ff q = two_prod(r0, r0);                      // r0^2 exactly
  ff m = ff_mul(x, q);                          // x r0^2 ~ 1
  float delta = __fsub_rn(__fsub_rn(1.f, m.hi), m.lo);
  return fast_two_sum(r0, 0.5f * r0 * delta);
}

}  // namespace fpt
