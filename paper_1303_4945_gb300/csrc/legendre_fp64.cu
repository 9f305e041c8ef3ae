// legendre_fp64.cu -- Legendre stage (Eqs. syn2 and ana1) in IEEE double.
//
// One thread owns one north/south ring pair and walks l upwards from
// l0 = max(m, |s|), generating sLambda_lm on the fly by the three-term recursion
// of Sect. 4.1 and applying each value as soon as it exists (the fused loop of
// Sect. 3.2, Figs. 1-2).  The southern ring of a pair comes for free from
//   sLambda_lm(pi - t) = (-1)^(l+m) (-s)Lambda_lm(t):
// even and odd (l+m) terms are kept apart and combined at the end.
//
// Spin s != 0 runs the +s and -s recursions side by side, each with its own
// exponent, and contracts them with P = E + iB and M = E - iB:
//   Q + iU = sum_m e^{im phi} [ -(1/2) sum_l (P (s)Lambda + (-1)^s M (-s)Lambda) ] + c.c. terms,
// see leg_syn_spin; the analysis uses W+- = G_Q +- i G_U the same way.
// Blocks of the growth phase in which no lane has reached scale 0 run the
// recursion alone.
//
// Enhanced exponent range (Sect. 4.1): the recursion pair is held as
// y * 2^(600 scale); while scale < 0 the terms are below ~2^-300 and are not
// accumulated; every 8 steps values above 2^300 are scaled down by 2^-600.
#include "sht_device.cuh"

namespace sht {

struct LegArgs {
  int lmax, spin, npairs, nm, astride;
  const int *mval;
  const int64_t *mstart;
  const int64_t *coef_off;
  const Coef *coef;
  const double2 *pm;  // spin: P = E + iB, M = E - iB per (array, m, l), indexed like coef
  int64_t ncoef;      // pm's entries per array
  const double2 *mpre;
  const PairDev *pairs;
  DevPtrs alm;
  double2 *phase;  // [nmaps][nm][npairs][2]
  const int2 *syn_items;
  const int4 *ana_items;
  const int64_t *part_off;
  double *part;
  int ppt, add;
  int ptr_off;  // batch: first entry of this plan in the pointer table
  int real;     // real-harmonic storage of the a_lm (spin-0 synthesis reads them directly)
  int half;     // m > 0 coefficients count half (SHT_GRADIENT with the adjoint analysis)
};

__device__ __forceinline__ int warp_any(bool b) { return __any_sync(0xffffffffu, b); }

// ---------------------------------------------------------------------------
// Synthesis, spin 0:  F_{m,y} = sum_l a_lm lambda_lm(theta_y)   (Eq. syn2)
// ---------------------------------------------------------------------------
template <int NJ>
__device__ __forceinline__ void leg_syn_s0_body(const LegArgs &a, double *const *ptrs, const int2 item) {
  const int mi = item.x;
  const int p = item.y + threadIdx.x;
  const bool valid = p < a.npairs;
  const int m = a.mval[mi];
  const int l0 = m, lmax = a.lmax;
  const Coef *__restrict__ cf = a.coef + a.coef_off[mi] - l0;
  const int64_t st = a.astride;
  const double2 *al[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) al[j] = reinterpret_cast<const double2 *>(ptrs[j]) + a.mstart[mi];

  const PairDev pd = a.pairs[valid ? p : 0];
  const double x = pd.x;
  double mant;
  int E, scale;
  start_value(m, 0, pd, a.mpre[mi], &mant, &E);
  double lc = valid ? to_scaled(mant, E, &scale) : 0.0;
  if (!valid) scale = 0;
  double lp = 0.0;
  double acc[2][NJ][2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[q][j][0] = acc[q][j][1] = 0.0;

  int l = l0;
  // growth phase: 8 steps per check, terms accumulate only at scale 0
  // (values at scale < 0 are below 2^-250); blocks in which no lane of the
  // warp has reached scale 0 run the recursion alone
  while (l <= lmax && warp_any(scale < 0)) {
    if (!warp_any(scale == 0)) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (l <= lmax) {
          const Coef c = ldg_coef(cf + l);
          const double ln = fma(c.a * x, lc, -c.c * lp);
          lp = lc;
          lc = ln;
          ++l;
        }
      }
      if (scale < 0 && fabs(lc) > kScaleUp) {
        lc *= kScaleFactor;
        lp *= kScaleFactor;
        ++scale;
      }
      continue;
    }
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        if (l <= lmax) {
          const double w = (scale == 0) ? lc : 0.0;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const double2 av = __ldg(al[j] + l * st);
            acc[par][j][0] = fma(av.x, w, acc[par][j][0]);
            acc[par][j][1] = fma(av.y, w, acc[par][j][1]);
          }
          const Coef c = ldg_coef(cf + l);
          const double ln = fma(c.a * x, lc, -c.c * lp);
          lp = lc;
          lc = ln;
          ++l;
        }
      }
    }
    if (scale < 0 && fabs(lc) > kScaleUp) {
      lc *= kScaleFactor;
      lp *= kScaleFactor;
      ++scale;
    }
  }
  // all lanes of the warp active: plain fused loop (offset l - l0 is even here)
  for (; l + 1 <= lmax; l += 2) {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      const int ll = l + par;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const double2 av = __ldg(al[j] + ll * st);
        acc[par][j][0] = fma(av.x, lc, acc[par][j][0]);
        acc[par][j][1] = fma(av.y, lc, acc[par][j][1]);
      }
      const Coef c = ldg_coef(cf + ll);
      const double ln = fma(c.a * x, lc, -c.c * lp);
      lp = lc;
      lc = ln;
    }
  }
  if (l <= lmax) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double2 av = __ldg(al[j] + l * st);
      acc[0][j][0] = fma(av.x, lc, acc[0][j][0]);
      acc[0][j][1] = fma(av.y, lc, acc[0][j][1]);
    }
  }
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    double2 fn = make_double2(acc[0][j][0] + acc[1][j][0], acc[0][j][1] + acc[1][j][1]);
    double2 fs = make_double2(acc[0][j][0] - acc[1][j][0], acc[0][j][1] - acc[1][j][1]);
    if (m == 0) fn.y = fs.y = 0.0;  // Im a_l0 is ignored: the field is real
    if (a.real && m > 0) {  // stored [a_{l,m}, a_{l,-m}] = sqrt2 (Re a_lm, -Im a_lm): same factors for all l
      const double r = 0.70710678118654752440;
      fn = make_double2(fn.x * r, -fn.y * r);
      fs = make_double2(fs.x * r, -fs.y * r);
    }
    if (a.half && m > 0) {  // the sum is linear in the a_lm: halving them halves F_m
      fn = make_double2(0.5 * fn.x, 0.5 * fn.y);
      fs = make_double2(0.5 * fs.x, 0.5 * fs.y);
    }
    double2 *o = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
    o[0] = fn;
    o[1] = fs;
  }
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) leg_syn_s0(LegArgs a) {
  leg_syn_s0_body<NJ>(a, a.alm.p, a.syn_items[blockIdx.x]);
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) leg_syn_s0_batch(const LegArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const LegArgs &a = args[it.w];
  leg_syn_s0_body<NJ>(a, tbl.p + a.ptr_off, make_int2(it.x, it.y));
}

// ---------------------------------------------------------------------------
// Synthesis, spin s.  The +s and -s recursions run separately, each with its
// own exponent (near the poles one is smaller than the other by
// tan^{2s}(theta/2); mixing them in one variable would lose the small one).
// With P = E + iB and M = E - iB (tabulated per (m, l) before the launch):
//   north:  q = -(N1 + sig N2)/2,  u = -(-i N1 + i sig N2)/2,   N1 = sum P l+, N2 = sum M l-
//   south:  q = -(S3 + sig S4)/2,  u = -(-i S3 + i sig S4)/2,   S3 = sum (-1)^(l+m) P l-,
//                                                              S4 = sum (-1)^(l+m) M l+
// with sig = (-1)^s, from sLambda(pi - t) = (-1)^(l+m) (-s)Lambda(t).
// ---------------------------------------------------------------------------
template <int NJ>
__device__ __forceinline__ void leg_syn_spin_body(const LegArgs &a, double *const *ptrs, const int2 item) {
  const int mi = item.x;
  const int p = item.y + threadIdx.x;
  const bool valid = p < a.npairs;
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax;
  const int64_t co = a.coef_off[mi] - l0;
  const Coef *__restrict__ cf = a.coef + co;
  const PairDev pd = a.pairs[valid ? p : 0];
  const double x = pd.x;
  double m1, m2;
  int e1, e2, scp, scm;
  start_value(m, s, pd, a.mpre[mi], &m1, &e1);
  start_value(m, -s, pd, a.mpre[mi], &m2, &e2);
  double lpc = valid ? to_scaled(m1, e1, &scp) : 0.0, lpp = 0.0;
  double lmc = valid ? to_scaled(m2, e2, &scm) : 0.0, lmp = 0.0;
  if (!valid) scp = scm = 0;
  double n1[NJ][2], n2[NJ][2], s3[NJ][2], s4[NJ][2];
#pragma unroll
  for (int j = 0; j < NJ; ++j) n1[j][0] = n1[j][1] = n2[j][0] = n2[j][1] = s3[j][0] = s3[j][1] = s4[j][0] = s4[j][1] = 0.0;

  auto step = [&](int l, int par, bool act) {
    const double wp = (act || scp == 0) ? lpc : 0.0;
    const double wm = (act || scm == 0) ? lmc : 0.0;
    const double sp = par ? -wp : wp, sm = par ? -wm : wm;  // (-1)^(l - l0) for the south ring
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double2 P = __ldg(a.pm + (int64_t)(2 * j) * a.ncoef + co + l);
      const double2 M = __ldg(a.pm + (int64_t)(2 * j + 1) * a.ncoef + co + l);
      n1[j][0] = fma(P.x, wp, n1[j][0]);
      n1[j][1] = fma(P.y, wp, n1[j][1]);
      n2[j][0] = fma(M.x, wm, n2[j][0]);
      n2[j][1] = fma(M.y, wm, n2[j][1]);
      s3[j][0] = fma(P.x, sm, s3[j][0]);
      s3[j][1] = fma(P.y, sm, s3[j][1]);
      s4[j][0] = fma(M.x, sp, s4[j][0]);
      s4[j][1] = fma(M.y, sp, s4[j][1]);
    }
    const Coef c = ldg_coef(cf + l);
    const double u = fma(c.a, x, c.ak), v = fma(c.a, x, -c.ak);  // A x +- AK, one rounding each
    const double np_ = fma(u, lpc, -c.c * lpp);
    const double nm_ = fma(v, lmc, -c.c * lmp);
    lpp = lpc;
    lpc = np_;
    lmp = lmc;
    lmc = nm_;
  };

  int l = l0;
  while (l <= lmax && warp_any(scp < 0 || scm < 0)) {
    if (!warp_any(scp == 0 || scm == 0)) {  // every term of the warp below 2^-250
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (l <= lmax) {
          const Coef c = ldg_coef(cf + l);
          const double np_ = fma(fma(c.a, x, c.ak), lpc, -c.c * lpp);
          const double nm_ = fma(fma(c.a, x, -c.ak), lmc, -c.c * lmp);
          lpp = lpc;
          lpc = np_;
          lmp = lmc;
          lmc = nm_;
          ++l;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
#pragma unroll
        for (int par = 0; par < 2; ++par) {
          if (l <= lmax) {
            step(l, par, false);
            ++l;
          }
        }
      }
    }
    if (scp < 0 && fabs(lpc) > kScaleUp) {
      lpc *= kScaleFactor;
      lpp *= kScaleFactor;
      ++scp;
    }
    if (scm < 0 && fabs(lmc) > kScaleUp) {
      lmc *= kScaleFactor;
      lmp *= kScaleFactor;
      ++scm;
    }
  }
  for (; l + 1 <= lmax; l += 2) {
    step(l, 0, true);
    step(l + 1, 1, true);
  }
  if (l <= lmax) step(l, 0, true);
  if (!valid) return;

  const double sig = (as & 1) ? -1.0 : 1.0;
  const double h0 = ((l0 + m) & 1) ? -0.5 : 0.5;  // (-1)^(l0+m) / 2
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    // z1 = N1 + sig N2 (q), z2 = sig N2 - N1 (u = -(i/2) z2)
    const double ar = n1[j][0] + sig * n2[j][0], ai = n1[j][1] + sig * n2[j][1];
    const double br = sig * n2[j][0] - n1[j][0], bi = sig * n2[j][1] - n1[j][1];
    const double cr = s3[j][0] + sig * s4[j][0], ci = s3[j][1] + sig * s4[j][1];
    const double dr = sig * s4[j][0] - s3[j][0], di = sig * s4[j][1] - s3[j][1];
    double2 qn = make_double2(-0.5 * ar, -0.5 * ai);
    double2 un = make_double2(0.5 * bi, -0.5 * br);
    double2 qs = make_double2(-h0 * cr, -h0 * ci);
    double2 us = make_double2(h0 * di, -h0 * dr);
    if (m == 0) qn.y = qs.y = un.y = us.y = 0.0;
    double2 *oq = a.phase + (((size_t)(2 * j) * a.nm + mi) * a.npairs + p) * 2;
    double2 *ou = a.phase + (((size_t)(2 * j + 1) * a.nm + mi) * a.npairs + p) * 2;
    oq[0] = qn;
    oq[1] = qs;
    ou[0] = un;
    ou[1] = us;
  }
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) leg_syn_spin(LegArgs a) {
  leg_syn_spin_body<NJ>(a, a.alm.p, a.syn_items[blockIdx.x]);
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) leg_syn_spin_batch(const LegArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const LegArgs &a = args[it.w];
  leg_syn_spin_body<NJ>(a, tbl.p + a.ptr_off, make_int2(it.x, it.y));
}
// ---------------------------------------------------------------------------
// Analysis (Eq. ana1): a_lm = sum_y G_{m,y} lambda_lm(theta_y).
// A CTA handles one m and a tile of kAnaThreads * PPT ring pairs; each thread
// walks PPT pairs in lockstep.  Per chunk of LC = 32 / V degrees every thread
// holds 32 partial sums (V values per l); a warp reduce-scatter leaves the
// warp total of value v in lane v, the 4 warps are added through shared
// memory and the tile's sum goes to the partial buffer.  A second kernel
// adds the tiles in a fixed order (deterministic result).
// ---------------------------------------------------------------------------

// 32 values per lane -> lane v holds sum over the warp of value v
__device__ __forceinline__ double warp_reduce_scatter32(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const bool up = lane & 16;
    const double send = up ? v[i] : v[i + 16];
    const double keep = up ? v[i + 16] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool up = lane & 8;
    const double send = up ? v[i] : v[i + 8];
    const double keep = up ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 4;
    const double send = up ? v[i] : v[i + 4];
    const double keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 2;
    const double send = up ? v[i] : v[i + 2];
    const double keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  {
    const bool up = lane & 1;
    const double send = up ? v[0] : v[1];
    const double keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
  return v[0];
}

template <int NJ, int PPT>
__device__ __forceinline__ void leg_ana_s0_body(const LegArgs &a, double *const *ptrs, const int4 item) {
  constexpr int V = 2 * NJ, LC = 32 / V;
  __shared__ double red[kAnaThreads / 32][32];
  const int mi = item.x, tile = item.y;
  const int m = a.mval[mi];
  const int l0 = m, lmax = a.lmax, nl = lmax - l0 + 1;
  const Coef *__restrict__ cf = a.coef + a.coef_off[mi] - l0;
  double *outp = a.part + a.part_off[mi] + (int64_t)(item.z >> 8) * nl * V;  // this item's slot

  double x[PPT], lc[PPT], lp[PPT];
  int scale[PPT];
  double ge[PPT][NJ][2], go[PPT][NJ][2];  // G_N + G_S, G_N - G_S
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = tile * (kAnaThreads * PPT) + threadIdx.x + k * kAnaThreads;
    const bool valid = p < a.npairs;
    const PairDev pd = a.pairs[valid ? p : 0];
    x[k] = pd.x;
    double mant;
    int E;
    start_value(m, 0, pd, a.mpre[mi], &mant, &E);
    lc[k] = valid ? to_scaled(mant, E, &scale[k]) : 0.0;
    if (!valid) scale[k] = 0;
    lp[k] = 0.0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      double2 gn = make_double2(0, 0), gs = make_double2(0, 0);
      if (valid) {
        const double2 *g = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
        gn = g[0];
        if (pd.south) gs = g[1];
      }
      ge[k][j][0] = gn.x + gs.x;
      ge[k][j][1] = gn.y + gs.y;
      go[k][j][0] = gn.x - gs.x;
      go[k][j][1] = gn.y - gs.y;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lb = l0; lb <= lmax; lb += LC) {
    bool mine = false;
#pragma unroll
    for (int k = 0; k < PPT; ++k) mine = mine || scale[k] == 0;
    if (!__syncthreads_or(mine)) {  // no term of this tile above 2^-250 yet: recursion only
#pragma unroll
      for (int q = 0; q < LC; ++q) {
        const int l = lb + q;
        if (l <= lmax) {
          const Coef c = ldg_coef(cf + l);
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const double ln = fma(c.a * x[k], lc[k], -c.c * lp[k]);
            lp[k] = lc[k];
            lc[k] = ln;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (scale[k] < 0 && fabs(lc[k]) > kScaleUp) {
          lc[k] *= kScaleFactor;
          lp[k] *= kScaleFactor;
          ++scale[k];
        }
      }
      if (warp == 0 && lb + lane / V <= lmax) outp[(int64_t)(lb - l0) * V + lane] = 0.0;
      continue;
    }
    double v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.0;
#pragma unroll
    for (int q = 0; q < LC; ++q) {
      const int l = lb + q;
      if (l <= lmax) {
        const Coef c = ldg_coef(cf + l);
        const bool even = ((l - l0) & 1) == 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const double w = (scale[k] == 0) ? lc[k] : 0.0;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const double gr = even ? ge[k][j][0] : go[k][j][0];
            const double gi = even ? ge[k][j][1] : go[k][j][1];
            v[q * V + 2 * j] = fma(w, gr, v[q * V + 2 * j]);
            v[q * V + 2 * j + 1] = fma(w, gi, v[q * V + 2 * j + 1]);
          }
          const double ln = fma(c.a * x[k], lc[k], -c.c * lp[k]);
          lp[k] = lc[k];
          lc[k] = ln;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (scale[k] < 0 && fabs(lc[k]) > kScaleUp) {
        lc[k] *= kScaleFactor;
        lp[k] *= kScaleFactor;
        ++scale[k];
      }
    }
    const double wsum = warp_reduce_scatter32(v);
    red[warp][lane] = wsum;
    __syncthreads();
    if (warp == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kAnaThreads / 32; ++w) t += red[w][lane];
      const int q = lane / V;
      if (lb + q <= lmax) outp[(int64_t)(lb - l0 + q) * V + (lane - q * V)] = t;
    }
    __syncthreads();
  }
}
template <int NJ, int PPT>
__global__ void __launch_bounds__(kAnaThreads) leg_ana_s0(LegArgs a) {
  leg_ana_s0_body<NJ, PPT>(a, a.alm.p, a.ana_items[blockIdx.x]);
}
template <int NJ, int PPT>
__global__ void __launch_bounds__(kAnaThreads) leg_ana_s0_batch(const LegArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const LegArgs &a = args[it.w];
  leg_ana_s0_body<NJ, PPT>(a, tbl.p + a.ptr_off, make_int4(it.x, it.y, it.z, 0));
}

// Spin analysis with separate +s / -s recursions.  Per ring W+ = GQ + i GU,
// W- = GQ - i GU; per degree l the pair contributes
//   T1 = W+_N l+ + (-1)^(l+m) W+_S l-,   T2 = W-_N l- + (-1)^(l+m) W-_S l+,
// and the reduction kernel forms E = -(T1 + sig T2)/2, B = -(i/2)(sig T2 - T1).
template <int NJ, int PPT>
__device__ __forceinline__ void leg_ana_spin_body(const LegArgs &a, double *const *ptrs, const int4 item) {
  constexpr int V = 4 * NJ, LC = 32 / V;
  __shared__ double red[kAnaThreads / 32][32];
  const int mi = item.x, tile = item.y;
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax, nl = lmax - l0 + 1;
  const Coef *__restrict__ cf = a.coef + a.coef_off[mi] - l0;
  double *outp = a.part + a.part_off[mi] + (int64_t)(item.z >> 8) * nl * V;  // this item's slot
  const double sg0 = ((l0 + m) & 1) ? -1.0 : 1.0;

  double x[PPT], lpc[PPT], lmc[PPT], lpp[PPT], lmp[PPT];
  int scp[PPT], scm[PPT];
  double wpn[PPT][NJ][2], wmn[PPT][NJ][2], wps[PPT][NJ][2], wms[PPT][NJ][2];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = tile * (kAnaThreads * PPT) + threadIdx.x + k * kAnaThreads;
    const bool valid = p < a.npairs;
    const PairDev pd = a.pairs[valid ? p : 0];
    x[k] = pd.x;
    double m1, m2;
    int e1, e2;
    start_value(m, s, pd, a.mpre[mi], &m1, &e1);
    start_value(m, -s, pd, a.mpre[mi], &m2, &e2);
    lpc[k] = valid ? to_scaled(m1, e1, &scp[k]) : 0.0;
    lmc[k] = valid ? to_scaled(m2, e2, &scm[k]) : 0.0;
    if (!valid) scp[k] = scm[k] = 0;
    lpp[k] = lmp[k] = 0.0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      double2 qn = make_double2(0, 0), qs = make_double2(0, 0), un = make_double2(0, 0), us = make_double2(0, 0);
      if (valid) {
        const double2 *gq = a.phase + (((size_t)(2 * j) * a.nm + mi) * a.npairs + p) * 2;
        const double2 *gu = a.phase + (((size_t)(2 * j + 1) * a.nm + mi) * a.npairs + p) * 2;
        qn = gq[0];
        un = gu[0];
        if (pd.south) {
          qs = gq[1];
          us = gu[1];
        }
      }
      // W+ = GQ + i GU, W- = GQ - i GU; the south ones carry (-1)^(l0+m)
      wpn[k][j][0] = qn.x - un.y;
      wpn[k][j][1] = qn.y + un.x;
      wmn[k][j][0] = qn.x + un.y;
      wmn[k][j][1] = qn.y - un.x;
      wps[k][j][0] = sg0 * (qs.x - us.y);
      wps[k][j][1] = sg0 * (qs.y + us.x);
      wms[k][j][0] = sg0 * (qs.x + us.y);
      wms[k][j][1] = sg0 * (qs.y - us.x);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lb = l0; lb <= lmax; lb += LC) {
    bool mine = false;
#pragma unroll
    for (int k = 0; k < PPT; ++k) mine = mine || scp[k] == 0 || scm[k] == 0;
    if (!__syncthreads_or(mine)) {  // no term of this tile above 2^-250 yet: recursion only
#pragma unroll
      for (int q = 0; q < LC; ++q) {
        const int l = lb + q;
        if (l <= lmax) {
          const Coef c = ldg_coef(cf + l);
#pragma unroll
          for (int k = 0; k < PPT; ++k) {
            const double np_ = fma(fma(c.a, x[k], c.ak), lpc[k], -c.c * lpp[k]);
            const double nm_ = fma(fma(c.a, x[k], -c.ak), lmc[k], -c.c * lmp[k]);
            lpp[k] = lpc[k];
            lpc[k] = np_;
            lmp[k] = lmc[k];
            lmc[k] = nm_;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (scp[k] < 0 && fabs(lpc[k]) > kScaleUp) {
          lpc[k] *= kScaleFactor;
          lpp[k] *= kScaleFactor;
          ++scp[k];
        }
        if (scm[k] < 0 && fabs(lmc[k]) > kScaleUp) {
          lmc[k] *= kScaleFactor;
          lmp[k] *= kScaleFactor;
          ++scm[k];
        }
      }
      if (warp == 0 && lb + lane / V <= lmax) outp[(int64_t)(lb - l0) * V + lane] = 0.0;
      continue;
    }
    double v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.0;
#pragma unroll
    for (int q = 0; q < LC; ++q) {
      const int l = lb + q;
      if (l <= lmax) {
        const Coef c = ldg_coef(cf + l);
        const bool even = ((l - l0) & 1) == 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          const double wp = (scp[k] == 0) ? lpc[k] : 0.0;
          const double wm = (scm[k] == 0) ? lmc[k] : 0.0;
          const double sp = even ? wp : -wp, sm = even ? wm : -wm;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const int o = q * V + 4 * j;
            v[o + 0] = fma(wp, wpn[k][j][0], fma(sm, wps[k][j][0], v[o + 0]));
            v[o + 1] = fma(wp, wpn[k][j][1], fma(sm, wps[k][j][1], v[o + 1]));
            v[o + 2] = fma(wm, wmn[k][j][0], fma(sp, wms[k][j][0], v[o + 2]));
            v[o + 3] = fma(wm, wmn[k][j][1], fma(sp, wms[k][j][1], v[o + 3]));
          }
          const double u = fma(c.a, x[k], c.ak), w = fma(c.a, x[k], -c.ak);  // A x +- AK, one rounding each
          const double np_ = fma(u, lpc[k], -c.c * lpp[k]);
          const double nm_ = fma(w, lmc[k], -c.c * lmp[k]);
          lpp[k] = lpc[k];
          lpc[k] = np_;
          lmp[k] = lmc[k];
          lmc[k] = nm_;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (scp[k] < 0 && fabs(lpc[k]) > kScaleUp) {
        lpc[k] *= kScaleFactor;
        lpp[k] *= kScaleFactor;
        ++scp[k];
      }
      if (scm[k] < 0 && fabs(lmc[k]) > kScaleUp) {
        lmc[k] *= kScaleFactor;
        lmp[k] *= kScaleFactor;
        ++scm[k];
      }
    }
    const double wsum = warp_reduce_scatter32(v);
    red[warp][lane] = wsum;
    __syncthreads();
    if (warp == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kAnaThreads / 32; ++w) t += red[w][lane];
      const int q = lane / V;
      if (lb + q <= lmax) outp[(int64_t)(lb - l0) * V + lane] = t;
    }
    __syncthreads();
  }
}
template <int NJ, int PPT>
__global__ void __launch_bounds__(kAnaThreads) leg_ana_spin(LegArgs a) {
  leg_ana_spin_body<NJ, PPT>(a, a.alm.p, a.ana_items[blockIdx.x]);
}
template <int NJ, int PPT>
__global__ void __launch_bounds__(kAnaThreads) leg_ana_spin_batch(const LegArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const LegArgs &a = args[it.w];
  leg_ana_spin_body<NJ, PPT>(a, tbl.p + a.ptr_off, make_int4(it.x, it.y, it.z, 0));
}

// Adds the tiles of every (m, l) in tile order and writes a_lm.
// spin 0: V = 2 njobs values (re, im per job).
// spin s: V = 4 njobs values (T1, T2 per job): E = -(T1 + sig T2)/2, B = -(i/2)(sig T2 - T1).
__global__ void ana_reduce(int lmax, int spin, int nm, int njobs_pad, int ncomp, int astride, int add,
                           int real, int grad,
                           const int *__restrict__ mval, const int64_t *__restrict__ mstart,
                           const int64_t *__restrict__ part_off, const int *__restrict__ nslot,
                           const double *__restrict__ part, DevPtrs alm) {
  const int mi = blockIdx.y;
  const int m = mval[mi];
  const int as = spin < 0 ? -spin : spin;
  const int l0 = m > as ? m : as;
  const int nl = lmax - l0 + 1;
  const int V = (spin ? 4 : 2) * njobs_pad;
  const int l = l0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  const int nt = nslot[mi];
  const double *pb = part + part_off[mi] + (int64_t)(l - l0) * V;
  const int64_t idx = mstart[mi] + (int64_t)l * astride;
  const int vper = spin ? 4 : 2;
  for (int j = 0; j < ncomp; ++j) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int tt = 0; tt < nt; ++tt)
      for (int k = 0; k < vper; ++k) t[k] += pb[(int64_t)tt * nl * V + vper * j + k];
    double2 out[2];
    int nout;
    if (spin == 0) {
      out[0] = make_double2(t[0], m == 0 ? 0.0 : t[1]);
      nout = 1;
    } else {
      const double sig = (as & 1) ? -1.0 : 1.0;
      out[0] = make_double2(-0.5 * (t[0] + sig * t[2]), -0.5 * (t[1] + sig * t[3]));
      const double zr = sig * t[2] - t[0], zi = sig * t[3] - t[1];
      out[1] = make_double2(0.5 * zi, -0.5 * zr);
      if (m == 0) out[0].y = out[1].y = 0.0;
      nout = 2;
    }
    for (int c = 0; c < nout; ++c) {
      double2 *o = reinterpret_cast<double2 *>(alm.p[nout * j + c]) + idx;
      double2 r = (real && m > 0) ? complex_to_real(out[c]) : out[c];
      if (grad && m > 0) r = make_double2(2.0 * r.x, 2.0 * r.y);  // the stored a_lm also stands for a_{l,-m}
      if (add) {
        const double2 old = *o;
        r.x += old.x;
        r.y += old.y;
      }
      *o = r;
    }
  }
  // spin: entries l < |s| (outside the recursion) are zero for l >= m
  if (spin && l == l0 && !add) {
    for (int ll = m; ll < l0; ++ll) {
      const int64_t i2 = mstart[mi] + (int64_t)ll * astride;
      for (int j = 0; j < 2 * ncomp; ++j) reinterpret_cast<double2 *>(alm.p[j])[i2] = make_double2(0.0, 0.0);
    }
  }
}

// P = E + iB, M = E - iB for every (m, l) of a spin plan, indexed like the coefficient table
__global__ void alm_to_pm(int lmax, int spin, int nm, int astride, const int *__restrict__ mval,
                          const int64_t *__restrict__ mstart, const int64_t *__restrict__ coef_off, int64_t ncoef,
                          DevPtrs alm, double2 *__restrict__ out, int mode) {
  const int mi = blockIdx.x, j = blockIdx.y;
  if (coef_off[mi] >= ncoef) return;  // beyond the table (a mixed plan's m above its FP64 columns)
  const int deriv = mode & kAlmDeriv, real = (mode & kAlmReal) && mval[mi] > 0;
  const int m = mval[mi];
  const double hf = ((mode & kAlmHalf) && m > 0) ? 0.5 : 1.0;
  const int as = spin < 0 ? -spin : spin;
  const int l0 = m > as ? m : as;
  // deriv (Sect. 4.3): E = sqrt(l(l+1)) a_lm of the spin-0 array j, B = 0
  const double2 *E = reinterpret_cast<const double2 *>(alm.p[deriv ? j : 2 * j]) + mstart[mi];
  const double2 *B = reinterpret_cast<const double2 *>(alm.p[deriv ? j : 2 * j + 1]) + mstart[mi];
  double2 *P = out + (int64_t)(2 * j) * ncoef + coef_off[mi] - l0;
  double2 *M = out + (int64_t)(2 * j + 1) * ncoef + coef_off[mi] - l0;
  for (int l = l0 + threadIdx.x; l <= lmax; l += blockDim.x) {
    double2 e = E[(int64_t)l * astride], b = B[(int64_t)l * astride];
    if (real) {
      e = real_to_complex(e);
      b = real_to_complex(b);
    }
    if (deriv) {
      const double f = sqrt((double)l * (double)(l + 1));
      e = make_double2(e.x * f, e.y * f);
      b = make_double2(0.0, 0.0);
    }
    if (m == 0) e.y = b.y = 0.0;  // Im of m = 0 coefficients is ignored
    e = make_double2(hf * e.x, hf * e.y);
    b = make_double2(hf * b.x, hf * b.y);
    P[l] = make_double2(e.x - b.y, e.y + b.x);
    M[l] = make_double2(e.x + b.y, e.y - b.x);
  }
}
// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static LegArgs make_args(const sht_plan_s *P, const DevPtrs &alm, int polar, bool lo = false) {
  LegArgs a;
  a.lmax = P->lmax;
  a.spin = P->spin;
  a.npairs = P->npairs;
  a.nm = P->nm;
  a.astride = P->astride;
  a.mval = P->d_mval;
  a.mstart = P->d_mstart;
  a.coef_off = P->d_coef_off;
  a.coef = P->d_coef;
  a.pm = P->d_pm64;
  a.ncoef = P->ncoef64;  // the P/M table's stride between arrays
  a.mpre = P->d_mpre;
  a.pairs = P->d_pairs;
  a.alm = alm;
  a.phase = P->d_phase;
  a.syn_items = lo ? P->d_syn_lo[polar] : P->d_syn_items[polar];
  a.ana_items = lo ? P->d_ana_lo[polar] : P->d_ana_items[polar];
  a.part_off = P->d_ana_part_off[polar];
  a.part = P->d_part;
  a.ppt = P->ana_ppt;
  a.add = 0;
  a.real = 0;
  a.half = 0;
  return a;
}

// Legendre stage over an explicit work list (stage 0: synthesis items int2, 1:
// analysis items int4); no a_lm conversion (launch_alm_prepare_fp64 does it)
cudaError_t launch_leg_fp64_items(const sht_plan_s *P, int stage, const DevPtrs &alm, int polar, const void *items,
                                  int n, cudaStream_t st, int amode) {
  if (n == 0) return cudaSuccess;
  LegArgs a = make_args(P, alm, polar);
  a.real = (amode & kAlmReal) ? 1 : 0;
  a.half = (amode & kAlmHalf) ? 1 : 0;
  const int nj = P->njobs_pad;
  if (stage == 0) {
    a.syn_items = static_cast<const int2 *>(items);
    if (P->spin == 0) {
      switch (nj) {
        case 1: leg_syn_s0<1><<<n, kSynTile, 0, st>>>(a); break;
        case 2: leg_syn_s0<2><<<n, kSynTile, 0, st>>>(a); break;
        case 4: leg_syn_s0<4><<<n, kSynTile, 0, st>>>(a); break;
        case 8: leg_syn_s0<8><<<n, kSynTile, 0, st>>>(a); break;
        default: leg_syn_s0<16><<<n, kSynTile, 0, st>>>(a); break;
      }
    } else {
      switch (nj) {
        case 1: leg_syn_spin<1><<<n, kSynTile, 0, st>>>(a); break;
        case 2: leg_syn_spin<2><<<n, kSynTile, 0, st>>>(a); break;
        case 4: leg_syn_spin<4><<<n, kSynTile, 0, st>>>(a); break;
        default: leg_syn_spin<8><<<n, kSynTile, 0, st>>>(a); break;
      }
    }
  } else {
    a.ana_items = static_cast<const int4 *>(items);
    if (P->spin == 0)
      ana_shape_s0(nj, P->ana_ppt, [&](auto sh) {
        leg_ana_s0<decltype(sh)::nj, decltype(sh)::ppt><<<n, kAnaThreads, 0, st>>>(a);
      });
    else
      ana_shape_spin(nj, P->ana_ppt, [&](auto sh) {
        leg_ana_spin<decltype(sh)::nj, decltype(sh)::ppt><<<n, kAnaThreads, 0, st>>>(a);
      });
  }
  return cudaGetLastError();
}

cudaError_t launch_leg_syn_fp64(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st, bool lo,
                                int mode) {
  const int n = lo ? P->nsyn_lo[polar] : P->nsyn_items[polar];
  if (n == 0) return cudaSuccess;
  cudaError_t e = launch_alm_prepare_fp64(P, alm, st, mode);
  if (e != cudaSuccess) return e;
  return launch_leg_fp64_items(P, 0, alm, polar, lo ? (const void *)P->d_syn_lo[polar] : P->d_syn_items[polar], n,
                               st, mode);
}

cudaError_t launch_leg_ana_fp64(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st, bool lo) {
  const int n = lo ? P->nana_lo[polar] : P->nana_items[polar];
  return launch_leg_fp64_items(P, 1, alm, polar, lo ? (const void *)P->d_ana_lo[polar] : P->d_ana_items[polar], n,
                               st);
}

cudaError_t launch_ana_reduce(const sht_plan_s *P, const DevPtrs &alm, int polar, int add, cudaStream_t st,
                              bool real, bool grad) {
  dim3 grid((P->lmax + 1 + 127) / 128, P->nm);
  ana_reduce<<<grid, 128, 0, st>>>(P->lmax, P->spin, P->nm, P->njobs_pad, P->ncomp, P->astride, add,
                                   real ? 1 : 0, grad ? 1 : 0,
                                   P->d_mval, P->d_mstart, P->d_ana_part_off[polar], P->d_ana_nslot[polar],
                                   P->d_part, alm);
  return cudaGetLastError();
}

}  // namespace sht

// ---------------------------------------------------------------------------
// batches (sht_batch_execute): per-plan argument records and batched launches
// ---------------------------------------------------------------------------
namespace sht {

size_t leg_fp64_args_size() { return sizeof(LegArgs); }

void leg_fp64_fill_args(const sht_plan_s *P, int polar, int ptr_off, void *out, bool lo) {
  DevPtrs none;
  memset(&none, 0, sizeof(none));
  LegArgs a = make_args(P, none, polar, lo);
  a.ptr_off = ptr_off;
  memcpy(out, &a, sizeof(a));
}

cudaError_t launch_alm_prepare_fp64(const sht_plan_s *P, const DevPtrs &alm, cudaStream_t st, int mode) {
  if (P->spin == 0 || P->nm == 0) return cudaSuccess;
  dim3 g(P->nm, P->njobs_pad);
  alm_to_pm<<<g, 256, 0, st>>>(P->lmax, P->spin, P->nm, P->astride, P->d_mval, P->d_mstart, P->d_coef_off,
                               P->ncoef64, alm, P->d_pm64, mode);
  return cudaGetLastError();
}

// stage 0: synthesis, 1: analysis; all plans of the launch share spin class, njobs_pad and tiling
cudaError_t launch_leg_fp64_batch(int stage, int spin, int nj, int ppt, const void *args, const int4 *items,
                                  int n, const PtrTable &tbl, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const LegArgs *a = static_cast<const LegArgs *>(args);
  if (stage == 0) {
    if (spin == 0) {
      switch (nj) {
        case 1: leg_syn_s0_batch<1><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 2: leg_syn_s0_batch<2><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 4: leg_syn_s0_batch<4><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 8: leg_syn_s0_batch<8><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        default: leg_syn_s0_batch<16><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
      }
    } else {
      switch (nj) {
        case 1: leg_syn_spin_batch<1><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 2: leg_syn_spin_batch<2><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 4: leg_syn_spin_batch<4><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        default: leg_syn_spin_batch<8><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
      }
    }
  } else {
    if (spin == 0)
      ana_shape_s0(nj, ppt, [&](auto sh) {
        leg_ana_s0_batch<decltype(sh)::nj, decltype(sh)::ppt><<<n, kAnaThreads, 0, st>>>(a, items, tbl);
      });
    else
      ana_shape_spin(nj, ppt, [&](auto sh) {
        leg_ana_spin_batch<decltype(sh)::nj, decltype(sh)::ppt><<<n, kAnaThreads, 0, st>>>(a, items, tbl);
      });
  }
  return cudaGetLastError();
}

}  // namespace sht
