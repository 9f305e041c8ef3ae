// df.cuh -- double-float arithmetic: a value held as hi + lo, two FP32 numbers.
//
// On GB300 the FP32 pipe issues 64 times the FP64 rate, so the mixed form runs
// its inner loops on FP32 pairs.  Products use the exact FMA split (Dekker /
// Kahan two-product), sums Knuth's two-sum; about 46 significant bits survive
// per operation.  No contraction: every step is an explicit *_rn intrinsic.
// Values must lie in FP32's exponent range (the low word keeps full relative
// precision for magnitudes above about 1e-30).
#pragma once

namespace sht {

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 f2_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double f2_val(f2 a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // needs |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a * b as an unevaluated pair
__device__ __forceinline__ f2 mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}
__device__ __forceinline__ f2 neg(f2 a) { return {-a.h, -a.l}; }

// a b + c d, normalised.  The final fast two-sum is needed: when the
// recursion's terms cancel (oscillatory regime) the low word of the raw sum
// can be as large as the high word, and the next product would then drop
// bits at FP32 precision.
__device__ __forceinline__ f2 dot2(f2 a, f2 b, f2 c, f2 d) {
  const f2 p = mul(a, b), q = mul(c, d);
  const f2 s = two_sum(p.h, q.h);
  return fast_two_sum(s.h, __fadd_rn(__fadd_rn(p.l, q.l), s.l));
}
__device__ __forceinline__ void renorm(f2 &a) { a = fast_two_sum(a.h, a.l); }
// a + b with the low word carried unnormalised (a running sum of a few dozen
// terms: the low word stays within a few ulps of the high word's last bit)
__device__ __forceinline__ f2 f2_add_lazy(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return {s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l)};
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l));
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) { return f2_add(a, neg(b)); }

}  // namespace sht
