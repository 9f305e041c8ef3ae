// tables.cu -- plan-time kernels: recursion coefficients and start-value prefactors.
//
// Recursion of Sect. 4.1 (the Wigner-d recursion it takes from Kostelec &
// Rockmore), restated for d^l_{a b} with
// a = -m, b = s:
//   [cos t + m s / (l (l+1))] d^l = c1_l d^{l-1} + c2_l d^{l+1},
//   c1_l = sqrt((l^2 - m^2)(l^2 - s^2)) / (l (2l+1)),
//   c2_l = sqrt(((l+1)^2 - m^2)((l+1)^2 - s^2)) / ((l+1)(2l+1)).
// With lambda_l = (-1)^m N_l d^l, N_l = sqrt((2l+1)/(4 pi)), this becomes
//   lambda_{l+1} = (A_l cos t + AK_l) lambda_l - C_l lambda_{l-1},
//   A_l  = N_{l+1} / (N_l c2_l)  = (l+1) sqrt((2l+3)(2l+1)) / sqrt(((l+1)^2 - m^2)((l+1)^2 - s^2)),
//   AK_l = A_l m s / (l (l+1)),
//   C_l  = N_{l+1} c1_l / (N_{l-1} c2_l)
//        = sqrt((2l+3)/(2l-1)) (l+1)/l sqrt((l^2-m^2)(l^2-s^2) / (((l+1)^2-m^2)((l+1)^2-s^2))).
// For -s the same table applies with AK_l -> -AK_l.  For s = 0 these reduce to
// the familiar A_l = sqrt((4(l+1)^2 - 1)/((l+1)^2 - m^2)), C_l = A_l sqrt((l^2 - m^2)/(4 l^2 - 1)).
#include "sht_internal.h"

namespace sht {

// coef: the FP64 table's first ncoef64 entries (a mixed plan keeps only the prefix
// its FP64 columns read); coef32 (mixed plans): every entry
__global__ void coef_kernel(int lmax, int spin, int nm, const int *__restrict__ mval,
                            const int64_t *__restrict__ coef_off, Coef *__restrict__ coef, int64_t ncoef64,
                            float4 *__restrict__ coef32) {
  const int mi = blockIdx.x;
  if (mi >= nm) return;
  const int m = mval[mi];
  const int as = spin < 0 ? -spin : spin;
  const int l0 = m > as ? m : as;
  const double dm = m, ds = spin;
  for (int l = l0 + threadIdx.x; l <= lmax; l += blockDim.x) {
    const double L = l, L1 = l + 1.0;
    const double qa = (L1 * L1 - dm * dm), qb = (L1 * L1 - ds * ds);
    const double A = L1 * sqrt((2.0 * L + 3.0) * (2.0 * L + 1.0)) / (sqrt(qa) * sqrt(qb));
    const double AK = (l == 0) ? 0.0 : A * (dm * ds) / (L * L1);
    double C = 0.0;
    if (l > l0 && l > 0) {
      const double pa = (L * L - dm * dm), pb = (L * L - ds * ds);
      C = sqrt((2.0 * L + 3.0) / (2.0 * L - 1.0)) * (L1 / L) * sqrt(pa / qa) * sqrt(pb / qb);
    }
    const int64_t i = coef_off[mi] + (l - l0);
    if (i < ncoef64) coef[i] = Coef{A, AK, C, 0.0};
    if (coef32) {
      const float ah = (float)A, kh = (float)AK, ch = (float)C;
      coef32[2 * i] = make_float4(ah, (float)(A - (double)ah), kh, (float)(AK - (double)kh));
      coef32[2 * i + 1] = make_float4(ch, (float)(C - (double)ch), 0.f, 0.f);
    }
  }
}

// sqrt((2 l0 + 1)/(4 pi)) * sqrt((2 l0)! / ((l0 + k)! (l0 - k)!)) as (mantissa, exponent),
// k = s if m >= |s| else m.  The factorial ratio is a product of min(u, v)
// ratios (hi + j)/j accumulated in double-double with a separate exponent.
__global__ void prefactor_kernel(int spin, int nm, const int *__restrict__ mval, double2 *__restrict__ pre) {
  const int mi = blockIdx.x * blockDim.x + threadIdx.x;
  if (mi >= nm) return;
  const int m = mval[mi];
  const int as = spin < 0 ? -spin : spin;
  const int l0 = m > as ? m : as;
  const int k = (m >= as) ? as : m;
  const int u = l0 - k, v = l0 + k;  // (2 l0)! / (u! v!)
  double hi = 1.0, lo = 0.0;
  int ex = 0;
  for (int j = 1; j <= u; ++j) {
    const double num = (double)(v + j), den = (double)j;
    const double q = num / den;
    const double qe = fma(-q, den, num) / den;  // q + qe = num/den to ~1e-32
    const double p = hi * q;
    double e = fma(hi, q, -p) + (hi * qe + lo * q);
    hi = p + e;
    lo = e - (hi - p);
    int t;
    hi = frexp(hi, &t);
    lo = ldexp(lo, -t);
    ex += t;
  }
  // square root of (hi + lo) 2^ex
  if (ex & 1) {
    hi *= 2.0;
    lo *= 2.0;
    ex -= 1;
  }
  const double r = sqrt(hi);
  const double rl = (fma(-r, r, hi) + lo) / (2.0 * r);
  const double nrm = sqrt((2.0 * l0 + 1.0) / (4.0 * 3.14159265358979323846));
  double mant = (r + rl) * nrm;
  int t;
  mant = frexp(mant, &t);
  pre[mi] = make_double2(mant, (double)(ex / 2 + t));
}

cudaError_t launch_coef_tables(const sht_plan_s *P, cudaStream_t st) {
  if (P->nm > 0) {
    coef_kernel<<<P->nm, 256, 0, st>>>(P->lmax, P->spin, P->nm, P->d_mval, P->d_coef_off, P->d_coef, P->ncoef64,
                                       P->d_coef32);
    prefactor_kernel<<<(P->nm + 127) / 128, 128, 0, st>>>(P->spin, P->nm, P->d_mval, P->d_mpre);
  }
  return cudaGetLastError();
}

}  // namespace sht
