// sht_device.cuh -- device helpers shared by the Legendre kernels.
#pragma once
#include "sht_internal.h"

namespace sht {

__device__ __forceinline__ Coef ldg_coef(const Coef *p) {
  const double2 u = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return {u.x, u.y, v.x, v.y};
}

// ---- double-double pieces -------------------------------------------------
struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  double lo = s.lo + a.lo + b.lo;
  double hi = s.hi + lo;
  return {hi, lo - (hi - s.hi)};
}

// (hi, lo) * n for an integer n (|n| < 2^31)
__device__ __forceinline__ dd dd_mul_int(dd a, int n) {
  double dn = (double)n;
  double p = a.hi * dn;
  double e = fma(a.hi, dn, -p) + a.lo * dn;
  double hi = p + e;
  return {hi, e - (hi - p)};
}

// ---- start values (Sect. 4.1) ----------------------------------------------
//
// sLambda_{l0,m}(theta) = (-1)^m sqrt((2 l0 + 1)/(4 pi)) d^{l0}_{-m,s}(theta),
// l0 = max(m, |s|), where the lowest-order Wigner function is the single
// surviving term of Wigner's sum:
//   m >= |s| :  sqrt(R) cos^{m-s}(t/2) sin^{m+s}(t/2) = sqrt(R) 2^{m (log2 sin t - 1) + s log2 tan(t/2)}
//   s >  m   :  sqrt(R) cos^{s-m}(t/2) sin^{s+m}(t/2) = sqrt(R) 2^{s (log2 sin t - 1) + m log2 tan(t/2)}
//   -s > m   :  (-1)^{l0+m} sqrt(R) cos^{l0+m}(t/2) sin^{l0-m}(t/2)
//             = (-1)^{l0+m} sqrt(R) 2^{l0 (log2 sin t - 1) - m log2 tan(t/2)}
// with R = (2 l0)! / ((l0 + k)! (l0 - k)!).  The factor sqrt((2l0+1)/4pi) sqrt(R)
// is tabulated per m as (mantissa, exponent) in pre; the power of two is formed
// from log2 sin(theta) and log2 tan(theta/2) given in double-double, so the
// result carries ~1 ulp error whatever m is.
//
// Returns the value as mant * 2^E (mant = 0 for an exact zero).
__device__ __forceinline__ void start_value(int m, int s, const PairDev &pd, double2 pre,
                                            double *mant, int *E) {
  const int as = s < 0 ? -s : s;
  int l0, kap, neg = (m & 1);
  int qsin;  // power of sin(theta/2)
  if (m >= as) {
    l0 = m;
    kap = s;
    qsin = m + s;
  } else if (s > 0) {
    l0 = s;
    kap = m;
    qsin = s + m;
  } else {
    l0 = as;
    kap = -m;
    qsin = as - m;
    neg ^= ((as + m) & 1);
  }
  if (pd.pole) {  // theta = 0: cos(theta/2) = 1, sin(theta/2) = 0
    *mant = (qsin == 0) ? (neg ? -pre.x : pre.x) : 0.0;
    *E = (int)pre.y;
    return;
  }
  dd l1 = dd_add({pd.l1_hi, pd.l1_lo}, {-1.0, 0.0});
  dd L = dd_add(dd_mul_int(l1, l0), dd_mul_int({pd.l2_hi, pd.l2_lo}, kap));
  double fl = floor(L.hi);
  double f = (L.hi - fl) + L.lo;  // fractional part, in [-eps, 1 + eps)
  double v = exp2(f) * pre.x;
  *mant = neg ? -v : v;
  *E = (int)fl + (int)pre.y;
}

// value = mant * 2^E  ->  (y, scale) with value = y * 2^(kScaleStep * scale),
// y's exponent in [-kScaleStep/2, kScaleStep/2).
__device__ __forceinline__ double to_scaled(double mant, int E, int *scale) {
  if (mant == 0.0) {
    *scale = 0;
    return 0.0;
  }
  int sc = (E + kScaleStep / 2) >= 0 ? (E + kScaleStep / 2) / kScaleStep
                                     : -((-(E + kScaleStep / 2) + kScaleStep - 1) / kScaleStep);
  *scale = sc;
  return ldexp(mant, E - kScaleStep * sc);
}

// Analysis tilings the kernels are built for: f(AnaShape<NJ, PPT>{}) runs the
// instance for padded job count nj and ppt ring pairs per thread (the
// candidates the host offers per spin class; anything else maps to the default).
template <int NJ, int PPT>
struct AnaShape {
  static constexpr int nj = NJ, ppt = PPT;
};
template <class F>
inline void ana_shape_s0(int nj, int ppt, F &&f) {
  switch (nj) {
    case 1:
      if (ppt == 8) f(AnaShape<1, 8>{});
      else if (ppt == 2) f(AnaShape<1, 2>{});
      else if (ppt == 1) f(AnaShape<1, 1>{});  // the tensor-core analysis' tiling (its FP64 items)
      else f(AnaShape<1, 4>{});
      break;
    case 2:
      if (ppt == 2) f(AnaShape<2, 2>{});
      else if (ppt == 1) f(AnaShape<2, 1>{});
      else f(AnaShape<2, 4>{});
      break;
    case 4: f(AnaShape<4, 2>{}); break;
    case 8: f(AnaShape<8, 2>{}); break;
    default: f(AnaShape<16, 2>{}); break;
  }
}
template <class F>
inline void ana_shape_spin(int nj, int ppt, F &&f) {
  switch (nj) {
    case 1:
      if (ppt == 4) f(AnaShape<1, 4>{});
      else if (ppt == 1) f(AnaShape<1, 1>{});
      else f(AnaShape<1, 2>{});
      break;
    case 2: if (ppt == 1) f(AnaShape<2, 1>{}); else f(AnaShape<2, 2>{}); break;
    case 4: f(AnaShape<4, 2>{}); break;
    default: f(AnaShape<8, 2>{}); break;
  }
}

// Real-harmonic storage (Sect. 4.5; reading): for m > 0 the complex slot of a_lm
// holds [a_{l,m}, a_{l,-m}] = sqrt2 (Re a_lm, -Im a_lm), the coefficients of the
// real basis sqrt2 Re Y_lm, sqrt2 Im Y_lm; m = 0 entries are unchanged.
__device__ __forceinline__ double2 real_to_complex(double2 r) {
  const double h = 0.70710678118654752440;
  return make_double2(r.x * h, -r.y * h);
}
__device__ __forceinline__ double2 complex_to_real(double2 c) {
  const double q = 1.41421356237309504880;
  return make_double2(c.x * q, -c.y * q);
}

}  // namespace sht
