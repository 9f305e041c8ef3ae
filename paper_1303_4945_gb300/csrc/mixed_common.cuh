// mixed_common.cuh -- the double-float pieces of the mixed form's Legendre
// kernels (legendre_mixed.cu, legendre_tc.cu): three-float cos(theta), the
// exact products and normalised dot products of the recursion of Sect. 4.1, the
// enhanced exponent in steps of 2^104, the start values in pairs, and the
// kernels' argument record.
#pragma once
#include "df.cuh"
#include "sht_device.cuh"

namespace sht {

constexpr int kScaleStep32 = 104;
constexpr float kScaleUp32 = 0x1p+52f;
constexpr float kScaleFactor32 = 0x1p-104f;

// cos(theta) as three floats summing exactly to the FP64 value.  Next to the
// poles x = 1 - O(theta^2) and a two-float x would carry a fixed error of
// ~2^-48 that the recursion amplifies by ~l/theta; with three floats the
// mixed form evaluates at exactly the same x as the FP64 form.
struct f3 {
  float h, m, l;
};
__device__ __forceinline__ f3 f3_of(double v) {
  const float h = __double2float_rn(v);
  const double r = v - (double)h;
  const float m = __double2float_rn(r);
  return {h, m, __double2float_rn(r - (double)m)};
}
// a * x for a two-float a and a three-float x, as an unevaluated pair
__device__ __forceinline__ f2 mul(f2 a, f3 x) {
  const float p = __fmul_rn(a.h, x.h);
  float e = __fmaf_rn(a.h, x.h, -p);
  e = __fmaf_rn(a.h, x.l, e);
  e = __fmaf_rn(a.l, x.h, e);
  e = __fmaf_rn(a.h, x.m, e);
  return {p, e};
}
// a b + c d + e f, normalised (see dot2)
__device__ __forceinline__ f2 dot3(f2 a, f2 b, f2 c, f2 d, f2 e, f2 f) {
  const f2 p = mul(a, b), q = mul(c, d), r = mul(e, f);
  const f2 s1 = two_sum(p.h, q.h);
  const f2 s2 = two_sum(s1.h, r.h);
  return fast_two_sum(s2.h, __fadd_rn(__fadd_rn(__fadd_rn(p.l, q.l), r.l), __fadd_rn(s1.l, s2.l)));
}
// acc += w * a with a lazily carried low word (renormalised every few steps)
__device__ __forceinline__ void acc_mul(f2 &acc, f2 w, float ah, float al) {
  const f2 p = mul(w, f2{ah, al});
  const f2 s = two_sum(acc.h, p.h);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, p.l));
}
// Accumulation weight of a recursion value y held at the given scale.  The
// exponent is checked every 8 steps, so a value still labelled scale -1 may
// already have grown past the 2^52 threshold by up to the 8-step growth of
// the recursion (< 2^50): its true size y 2^-104 can reach 2^-2 and must be
// accumulated.  Values at scale <= -2 are below 2^(52+50-208) and are dropped.
__device__ __forceinline__ f2 weight(f2 y, int scale) {
  const float f = (scale == 0) ? 1.f : ((scale == -1) ? kScaleFactor32 : 0.f);
  return {y.h * f, y.l * f};
}

// True value below 2^-74 (scale -1: y 2^-104 with |y| < 2^30; scale <= -2:
// |y| < 2^102 between checks): even after two more steps (growth < 2^14) it
// stays below 2^-60 and its terms can be skipped.
__device__ __forceinline__ bool negligible(f2 y, int scale) {
  return scale <= -2 || (scale == -1 && fabsf(y.h) < 0x1p30f);
}

// (mant * 2^E) -> (y, scale) with value = y * 2^(104 scale), y's exponent in [-52, 52)
__device__ __forceinline__ f2 to_scaled32(double mant, int E, int *scale) {
  if (mant == 0.0) {
    *scale = 0;
    return {0.f, 0.f};
  }
  const int h = kScaleStep32 / 2;
  const int sc = (E + h) >= 0 ? (E + h) / kScaleStep32 : -((-(E + h) + kScaleStep32 - 1) / kScaleStep32);
  *scale = sc;
  return f2_of(ldexp(mant, E - kScaleStep32 * sc));
}

// Where a ring pair's terms start for one m: the first block of 16 degrees
// (counted from l0) that holds a degree pair whose values are not negligible
// (the test the kernels apply every second degree), and the recursion state at
// that block's first degree, as the kernels reach it (same steps, same rescale
// checks every eight degrees).  Kernels that walk the degrees in blocks of 16 let
// a pair join there with that state (before, it adds only terms below the
// negligible bound) and start a CTA at its pairs' earliest block.  lj = lmax + 1:
// the pair never contributes.  lexp: a power of two 2^lexp bounding the true
// size of every value the pair's recursion takes from its join block to lmax + 1
// (the tensor-core synthesis puts the pair's Lambda digits on that grid).  48
// bytes, read as three float4.
struct JoinRec {
  f2 lpc, lpp, lmc, lmp;  // +s current / previous, -s current / previous
  int scp, scm, lj, lexp;
};
static_assert(sizeof(JoinRec) == 48, "three float4");
__device__ __forceinline__ JoinRec ld_join(const float4 *p) {
  const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  JoinRec r;
  r.lpc = f2{a.x, a.y};
  r.lpp = f2{a.z, a.w};
  r.lmc = f2{b.x, b.y};
  r.lmp = f2{b.z, b.w};
  r.scp = __float_as_int(c.x);
  r.scm = __float_as_int(c.y);
  r.lj = __float_as_int(c.z);
  r.lexp = __float_as_int(c.w);
  return r;
}
constexpr int kJoinBlock = 16;  // degrees per join block

struct MixArgs {
  int lmax, spin, npairs, nm;
  const int *mval;
  const int64_t *coef_off;
  const float4 *coef32;  // per (m, l): {A.h, A.l, AK.h, AK.l}, {C.h, C.l, -, -}
  const float4 *alm32;   // [array][ncoef] {re.h, re.l, im.h, im.l}
  int64_t ncoef;
  const double2 *mpre;
  const PairDev *pairs;
  double2 *phase;
  const int2 *syn_items;
  const int4 *ana_items;
  const int64_t *part_off;
  double *part;
  int ptr_off;
  const float4 *join;  // JoinRec per (m index, pair), 3 float4 each
};

struct Coef32 {
  f2 a, ak, c;
};
__device__ __forceinline__ Coef32 ld_coef32(const float4 *p) {
  const float4 u = __ldg(p), v = __ldg(p + 1);
  return {{u.x, u.y}, {u.z, u.w}, {v.x, v.y}};
}

// spin-0 / spin start in the double-float representation
__device__ __forceinline__ void start_s0(int m, const PairDev &pd, double2 pre, f2 *lc, int *scale) {
  double mant;
  int E;
  start_value(m, 0, pd, pre, &mant, &E);
  *lc = to_scaled32(mant, E, scale);
}
__device__ __forceinline__ void start_s(int m, int s, const PairDev &pd, double2 pre, f2 *lc, int *scale) {
  double mant;
  int E;
  start_value(m, s, pd, pre, &mant, &E);
  *lc = to_scaled32(mant, E, scale);
}
}  // namespace sht
