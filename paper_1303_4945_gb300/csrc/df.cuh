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

// Conversions that keep off the FP64 pipe (it issues 1/64 of the FP32 rate, and
// conversions to or from FP64 run on it), for code whose inner loop is FP32.
//
// v as hi + lo from v's bit fields: hi = v truncated to 24 significant bits,
// lo = the remaining 29 bits rounded to FP32 (the 29-bit integer is made exact in
// two 2^23-offset halves, then scaled by powers of two: two steps below 2^-64 so
// that a low word under FP32's normal range rounds gradually).  |lo| < ulp(hi).
// |v| below 2^-126, FP32's normal range, gives a signed zero and |v| >= 2^128 an
// infinity (NaN stays NaN).  No path holds an FP64 instruction: a short rare path
// is predicated rather than branched, so it would be issued for every value.
__device__ __forceinline__ f2 f2_split(double v) {
  const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
  const unsigned e = (hw >> 20) & 0x7ffu, sign = hw & 0x80000000u;
  if (e - 897u > 253u) {
    if (e < 897u) return {__uint_as_float(sign), 0.0f};
    const bool nan = e == 2047u && ((hw & 0xfffffu) | lw) != 0u;
    return {__uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.0f};
  }
  const float h = __uint_as_float(sign | ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const unsigned r = lw & 0x1fffffffu;  // v - h in units of 2^(e - 1075)
  const float rh = __fsub_rn(__uint_as_float(0x4b000000u | (r >> 16)), 8388608.0f);
  const float rl = __fsub_rn(__uint_as_float(0x4b000000u | (r & 0xffffu)), 8388608.0f);
  const unsigned k = e < 1011u ? 64u : 0u;  // 2^(e - 1075) = 2^(e - 1075 + k) 2^-k
  const float l = __fmul_rn(__fmul_rn(__fmaf_rn(rh, 65536.0f, rl), __uint_as_float((e - 948u + k) << 23)),
                            __uint_as_float((127u - k) << 23));
  return {h, __uint_as_float(__float_as_uint(l) | sign)};
}
// x widened to double from its bit fields, all classes included (integer work only)
__device__ __forceinline__ double f2_widen(float x) {
  const unsigned b = __float_as_uint(x), sign = b & 0x80000000u, ef = (b >> 23) & 0xffu, mf = b & 0x7fffffu;
  unsigned hi, lo = mf << 29;
  if (ef - 1u <= 253u) {
    hi = sign | ((ef + 896u) << 20) | (mf >> 3);
  } else if (ef == 255u) {  // infinity, NaN
    hi = sign | 0x7ff00000u | (mf >> 3);
  } else if (mf == 0u) {
    hi = sign;
  } else {  // subnormal: mf 2^-149 with its top bit at p
    const unsigned p = 31u - __clz(mf);
    const unsigned long long frac = (unsigned long long)(mf ^ (1u << p)) << (52u - p);
    hi = sign | ((p + 874u) << 20) | (unsigned)(frac >> 32);
    lo = (unsigned)frac;
  }
  return __hiloint2double((int)hi, (int)lo);
}
// hi + lo as a double: two widenings on the bit fields, one FP64 addition
__device__ __forceinline__ double f2_join(f2 a) { return __dadd_rn(f2_widen(a.h), f2_widen(a.l)); }

}  // namespace sht
