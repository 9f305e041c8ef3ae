// legendre_mixed.cu -- Legendre stage (Eqs. syn2, ana1) in the mixed form.
//
// On GB300 the FP64 pipe issues 1/64 of the FP32 rate, so this form moves
// the whole inner loop (the recursion of Sect. 4.1 and the accumulation of
// Fig. 1 / Fig. 2) onto the FP32 pipe in compensated "double-float" pairs
// (value = hi + lo, two FP32 numbers).  Products use the exact FMA split
// (Dekker / Kahan two-product), sums Knuth's two-sum; about 46 significant
// bits survive per operation, enough for ~1e-12 after thousands of steps.
// FP64 remains for the recursion-coefficient tables, the start values and the
// conversion of inputs/outputs (the ring FFTs of mixed plans run the same
// double-float arithmetic, in fft.cu).
//
// Structure, ring pairing, parity split, the separate +s / -s recursions for
// spin and the analysis reduction follow legendre_fp64.cu; only the arithmetic
// type differs.  The enhanced exponent uses steps of 2^104: pairs above 2^52
// are scaled down every 8 steps; values at scale 0 and -1 are accumulated (the
// latter times 2^-104), anything smaller is negligible.  A mixed plan hands the
// items of small m near the poles to the FP64 kernels (sht_plan_s::fp64_m_below).
#include "mixed_common.cuh"

namespace sht {

// ---------------------------------------------------------------------------
// a_lm (FP64, user layout) -> double-float table indexed like the coefficients
// ---------------------------------------------------------------------------
__global__ void alm_to_f2(int lmax, int spin, int nm, int narr, int astride, const int *__restrict__ mval,
                          const int64_t *__restrict__ mstart, const int64_t *__restrict__ coef_off, int64_t ncoef,
                          DevPtrs alm, float4 *__restrict__ out, int mode) {
  const int mi = blockIdx.x;
  const int deriv = mode & kAlmDeriv, real = (mode & kAlmReal) && mval[mi] > 0;
  const int j = blockIdx.y;
  const int m = mval[mi];
  const double hf = ((mode & kAlmHalf) && m > 0) ? 0.5 : 1.0;
  const int as = spin < 0 ? -spin : spin;
  const int l0 = m > as ? m : as;
  if (spin == 0) {
    const double2 *src = reinterpret_cast<const double2 *>(alm.p[j]) + mstart[mi];
    float4 *dst = out + (int64_t)j * ncoef + coef_off[mi] - l0;
    for (int l = l0 + threadIdx.x; l <= lmax; l += blockDim.x) {
      double2 v = src[(int64_t)l * astride];
      if (real) v = real_to_complex(v);
      const f2 re = f2_of(hf * v.x), im = f2_of(hf * v.y);
      dst[l] = make_float4(re.h, re.l, im.h, im.l);
    }
    return;
  }
  // spin: P = E + iB and M = E - iB of job j (Im of m = 0 coefficients ignored);
  // deriv (Sect. 4.3): E = sqrt(l(l+1)) a_lm of the spin-0 array j, B = 0
  const double2 *E = reinterpret_cast<const double2 *>(alm.p[deriv ? j : 2 * j]) + mstart[mi];
  const double2 *B = reinterpret_cast<const double2 *>(alm.p[deriv ? j : 2 * j + 1]) + mstart[mi];
  float4 *P = out + (int64_t)(2 * j) * ncoef + coef_off[mi] - l0;
  float4 *M = out + (int64_t)(2 * j + 1) * ncoef + coef_off[mi] - l0;
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
    if (m == 0) e.y = b.y = 0.0;
    e = make_double2(hf * e.x, hf * e.y);
    b = make_double2(hf * b.x, hf * b.y);
    const f2 pr = f2_of(e.x - b.y), pi = f2_of(e.y + b.x), mr = f2_of(e.x + b.y), mi_ = f2_of(e.y - b.x);
    P[l] = make_float4(pr.h, pr.l, pi.h, pi.l);
    M[l] = make_float4(mr.h, mr.l, mi_.h, mi_.l);
  }
}

// ---------------------------------------------------------------------------
// synthesis, spin 0
//
// Loop bodies hold two steps (static even/odd parity) and are not unrolled
// further: the double-float step is ~170 instructions, and longer unrolled
// bodies stalled the issue on instruction fetch.
// ---------------------------------------------------------------------------
template <int NJ>
__device__ __forceinline__ void mix_syn_s0_body(const MixArgs &a, double *const *ptrs, const int2 item) {
  const int mi = item.x;
  const int p = item.y + threadIdx.x;
  const bool valid = p < a.npairs;
  const int m = a.mval[mi];
  const int l0 = m, lmax = a.lmax;
  const int64_t co = a.coef_off[mi] - l0;
  const float4 *__restrict__ cf = a.coef32 + 2 * co;
  const PairDev pd = a.pairs[valid ? p : 0];
  const f3 x = f3_of(pd.x);
  // zero until the pair joins at its join record's block (no terms, a recursion of zeros)
  f2 lc = {0.f, 0.f}, lp = {0.f, 0.f};
  int scale = 0;
  const float4 *jrec = a.join + ((size_t)mi * a.npairs + (valid ? p : 0)) * 3;
  const int lj = valid ? __float_as_int(__ldg(jrec + 2).z) : lmax + 1;
  f2 acc[2][NJ][2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[q][j][0] = acc[q][j][1] = f2{0.f, 0.f};

  auto step = [&](int l, int par, bool act) {
    const f2 w = act ? lc : weight(lc, scale);
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float4 v = __ldg(a.alm32 + (int64_t)j * a.ncoef + co + l);
      acc_mul(acc[par][j][0], w, v.x, v.y);
      acc_mul(acc[par][j][1], w, v.z, v.w);
    }
    const Coef32 c = ld_coef32(cf + 2 * l);
    const f2 t = mul(c.a, x);
    const f2 ln = dot2(t, lc, neg(c.c), lp);
    lp = lc;
    lc = ln;
  };
  auto recur = [&](int l) {  // recursion only (every lane's term negligible)
    const Coef32 c = ld_coef32(cf + 2 * l);
    const f2 t = mul(c.a, x);
    const f2 ln = dot2(t, lc, neg(c.c), lp);
    lp = lc;
    lc = ln;
  };
  auto renorm_all = [&]() {
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        renorm(acc[q][j][0]);
        renorm(acc[q][j][1]);
      }
  };

  // the warp starts at its lanes' earliest join block and walks carefully (scale
  // checks, negligible terms skipped) while a lane is below scale 0 or yet to join
  int l = __reduce_min_sync(0xffffffffu, lj);
  while (l <= lmax && __any_sync(0xffffffffu, scale < 0 || (lj <= lmax && lj >= l))) {
    if (lj == l) {
      const JoinRec r = ld_join(jrec);
      lc = r.lpc;
      lp = r.lpp;
      scale = r.scp;
    }
#pragma unroll 1
    for (int k = 0; k < 4 && l <= lmax; ++k, l += 2) {
      if (__all_sync(0xffffffffu, negligible(lc, scale))) {
        recur(l);
        if (l + 1 <= lmax) recur(l + 1);
      } else {
        step(l, 0, false);
        if (l + 1 <= lmax) step(l + 1, 1, false);
      }
    }
    if (scale < 0 && fabsf(lc.h) > kScaleUp32) {
      lc = {lc.h * kScaleFactor32, lc.l * kScaleFactor32};
      lp = {lp.h * kScaleFactor32, lp.l * kScaleFactor32};
      ++scale;
    }
    renorm_all();
  }
  int since = 0;
#pragma unroll 1
  for (; l + 1 <= lmax; l += 2) {
    step(l, 0, true);
    step(l + 1, 1, true);
    if (++since == 8) {
      renorm_all();
      since = 0;
    }
  }
  if (l <= lmax) step(l, 0, true);
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const double e0 = f2_val(acc[0][j][0]), e1 = f2_val(acc[0][j][1]);
    const double o0 = f2_val(acc[1][j][0]), o1 = f2_val(acc[1][j][1]);
    double2 fn = make_double2(e0 + o0, e1 + o1), fs = make_double2(e0 - o0, e1 - o1);
    if (m == 0) fn.y = fs.y = 0.0;
    double2 *o = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
    o[0] = fn;
    o[1] = fs;
  }
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) mix_syn_s0(MixArgs a) {
  mix_syn_s0_body<NJ>(a, nullptr, a.syn_items[blockIdx.x]);
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) mix_syn_s0_batch(const MixArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const MixArgs &a = args[it.w];
  mix_syn_s0_body<NJ>(a, tbl.p + a.ptr_off, make_int2(it.x, it.y));
}

// ---------------------------------------------------------------------------
// synthesis, spin s: separate +s / -s recursions (see legendre_fp64.cu)
// ---------------------------------------------------------------------------
template <int NJ>
__device__ __forceinline__ void mix_syn_spin_body(const MixArgs &a, double *const *ptrs, const int2 item) {
  const int mi = item.x;
  const int p = item.y + threadIdx.x;
  const bool valid = p < a.npairs;
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax;
  const int64_t co = a.coef_off[mi] - l0;
  const float4 *__restrict__ cf = a.coef32 + 2 * co;
  const PairDev pd = a.pairs[valid ? p : 0];
  const f3 x = f3_of(pd.x);
  // zero until the pair joins at its join record's block (no terms, a recursion of zeros)
  f2 lpc = {0.f, 0.f}, lmc = {0.f, 0.f}, lpp = {0.f, 0.f}, lmp = {0.f, 0.f};
  int scp = 0, scm = 0;
  const float4 *jrec = a.join + ((size_t)mi * a.npairs + (valid ? p : 0)) * 3;
  const int lj = valid ? __float_as_int(__ldg(jrec + 2).z) : lmax + 1;
  // N1 = sum P l+, N2 = sum M l-, S3 = sum (-1)^(l-l0) P l-, S4 = sum (-1)^(l-l0) M l+
  f2 r[NJ][4][2];
#pragma unroll
  for (int j = 0; j < NJ; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) r[j][k][0] = r[j][k][1] = f2{0.f, 0.f};

  auto step = [&](int l, int par, bool act) {
    const f2 wp = act ? lpc : weight(lpc, scp), wm = act ? lmc : weight(lmc, scm);
    const f2 sp = par ? neg(wp) : wp, sm = par ? neg(wm) : wm;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float4 P = __ldg(a.alm32 + (int64_t)(2 * j) * a.ncoef + co + l);
      const float4 M = __ldg(a.alm32 + (int64_t)(2 * j + 1) * a.ncoef + co + l);
      acc_mul(r[j][0][0], wp, P.x, P.y);
      acc_mul(r[j][0][1], wp, P.z, P.w);
      acc_mul(r[j][1][0], wm, M.x, M.y);
      acc_mul(r[j][1][1], wm, M.z, M.w);
      acc_mul(r[j][2][0], sm, P.x, P.y);
      acc_mul(r[j][2][1], sm, P.z, P.w);
      acc_mul(r[j][3][0], sp, M.x, M.y);
      acc_mul(r[j][3][1], sp, M.z, M.w);
    }
    const Coef32 c = ld_coef32(cf + 2 * l);
    const f2 t = mul(c.a, x);
    const f2 nc = neg(c.c);
    const f2 np_ = dot3(t, lpc, c.ak, lpc, nc, lpp);
    const f2 nm_ = dot3(t, lmc, neg(c.ak), lmc, nc, lmp);
    lpp = lpc;
    lpc = np_;
    lmp = lmc;
    lmc = nm_;
  };
  auto recur = [&](int l) {  // recursion only (every lane's terms negligible)
    const Coef32 c = ld_coef32(cf + 2 * l);
    const f2 t = mul(c.a, x);
    const f2 nc = neg(c.c);
    const f2 np_ = dot3(t, lpc, c.ak, lpc, nc, lpp);
    const f2 nm_ = dot3(t, lmc, neg(c.ak), lmc, nc, lmp);
    lpp = lpc;
    lpc = np_;
    lmp = lmc;
    lmc = nm_;
  };
  auto renorm_all = [&]() {
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        renorm(r[j][k][0]);
        renorm(r[j][k][1]);
      }
  };

  // the warp starts at its lanes' earliest join block and walks carefully (scale
  // checks, negligible terms skipped) while a lane is below scale 0 or yet to join
  int l = __reduce_min_sync(0xffffffffu, lj);
  while (l <= lmax && __any_sync(0xffffffffu, scp < 0 || scm < 0 || (lj <= lmax && lj >= l))) {
    if (lj == l) {
      const JoinRec r = ld_join(jrec);
      lpc = r.lpc;
      lpp = r.lpp;
      lmc = r.lmc;
      lmp = r.lmp;
      scp = r.scp;
      scm = r.scm;
    }
#pragma unroll 1
    for (int k = 0; k < 4 && l <= lmax; ++k, l += 2) {
      if (__all_sync(0xffffffffu, negligible(lpc, scp) && negligible(lmc, scm))) {
        recur(l);
        if (l + 1 <= lmax) recur(l + 1);
      } else {
        step(l, 0, false);
        if (l + 1 <= lmax) step(l + 1, 1, false);
      }
    }
    if (scp < 0 && fabsf(lpc.h) > kScaleUp32) {
      lpc = {lpc.h * kScaleFactor32, lpc.l * kScaleFactor32};
      lpp = {lpp.h * kScaleFactor32, lpp.l * kScaleFactor32};
      ++scp;
    }
    if (scm < 0 && fabsf(lmc.h) > kScaleUp32) {
      lmc = {lmc.h * kScaleFactor32, lmc.l * kScaleFactor32};
      lmp = {lmp.h * kScaleFactor32, lmp.l * kScaleFactor32};
      ++scm;
    }
    renorm_all();
  }
  int since = 0;
#pragma unroll 1
  for (; l + 1 <= lmax; l += 2) {
    step(l, 0, true);
    step(l + 1, 1, true);
    if (++since == 8) {
      renorm_all();
      since = 0;
    }
  }
  if (l <= lmax) step(l, 0, true);
  if (!valid) return;

  const double sig = (as & 1) ? -1.0 : 1.0;
  const double h0 = ((l0 + m) & 1) ? -0.5 : 0.5;
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const double n1r = f2_val(r[j][0][0]), n1i = f2_val(r[j][0][1]);
    const double n2r = f2_val(r[j][1][0]), n2i = f2_val(r[j][1][1]);
    const double s3r = f2_val(r[j][2][0]), s3i = f2_val(r[j][2][1]);
    const double s4r = f2_val(r[j][3][0]), s4i = f2_val(r[j][3][1]);
    const double ar = n1r + sig * n2r, ai = n1i + sig * n2i;
    const double br = sig * n2r - n1r, bi = sig * n2i - n1i;
    const double cr = s3r + sig * s4r, ci = s3i + sig * s4i;
    const double dr = sig * s4r - s3r, di = sig * s4i - s3i;
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
__global__ void __launch_bounds__(kSynTile) mix_syn_spin(MixArgs a) {
  mix_syn_spin_body<NJ>(a, nullptr, a.syn_items[blockIdx.x]);
}
template <int NJ>
__global__ void __launch_bounds__(kSynTile) mix_syn_spin_batch(const MixArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const MixArgs &a = args[it.w];
  mix_syn_spin_body<NJ>(a, tbl.p + a.ptr_off, make_int2(it.x, it.y));
}

// ---------------------------------------------------------------------------
// analysis (tiles and partial sums as in legendre_fp64.cu).
//
// Each thread walks PPT ring pairs.  For every degree l it sums its pairs'
// V contributions in registers and stores them to a shared-memory slot
// table [32 slots = LC degrees x V values][threads]; after LC degrees each warp
// sums its own 32 columns of the table (a warp's columns are written and read by
// that warp only: warp-level synchronisation), and after one CTA barrier warp 0
// adds the four warps' partials (double-buffered by chunk parity) to the item's
// slot of partial sums.  An
// item walks a group of consecutive tiles of one m tile after tile into one
// slot (the host sizes the groups), so the partials shrink by the group size.
// Degrees are walked two at a time so the even/odd parity is static.
// ---------------------------------------------------------------------------
template <int NJ, int PPT, bool SPIN>
__device__ __forceinline__ void mix_ana_body(const MixArgs &a, double *const *ptrs, const int4 item) {
  constexpr int V = (SPIN ? 4 : 2) * NJ, LC = 32 / V;
  static_assert(V * LC == 32, "32 slots per chunk");
  __shared__ f2 slot[32][kAnaThreads + 1];
  __shared__ f2 quart[2][kAnaThreads / 32][32];  // by chunk parity
  __shared__ int tstart[2][kAnaThreads / 32];     // per tile (parity): the warps' earliest join degree
  const int mi = item.x, ng = item.z & 255;  // ng tiles from tile item.y on, one slot of partial sums
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax, nl = lmax - l0 + 1;
  const float4 *__restrict__ cf = a.coef32 + 2 * (a.coef_off[mi] - l0);
  double *outp = a.part + a.part_off[mi] + (int64_t)(item.z >> 8) * nl * V;
  const double sg0 = ((l0 + m) & 1) ? -1.0 : 1.0;
  const int tid = threadIdx.x;

  // the group's tiles one after another; each adds its sums to the slot (the first
  // overwrites it), in a fixed order
#pragma unroll 1
  for (int gi = 0; gi < ng; ++gi) {
    const int tile = item.y + gi;
    f3 x[PPT];
    f2 lpc[PPT], lmc[PPT], lpp[PPT], lmp[PPT];
    int scp[PPT], scm[PPT];
    // the degree at which each pair's terms start (join record; zero state until then)
    int lj[PPT];
    // spin 0: g[k][j][0..1] = G_N + G_S, G_N - G_S (complex);
    // spin:   g[k][j][0..3] = W+_N, W-_N, (-1)^(l0+m) W+_S, (-1)^(l0+m) W-_S (complex)
    f2 g[PPT][NJ][SPIN ? 4 : 2][2];
    int jmin = lmax + 1;
  #pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int p = tile * (kAnaThreads * PPT) + tid + k * kAnaThreads;
      const bool valid = p < a.npairs;
      const PairDev pd = a.pairs[valid ? p : 0];
      x[k] = f3_of(pd.x);
      lj[k] = valid ? __float_as_int(__ldg(a.join + ((size_t)mi * a.npairs + p) * 3 + 2).z) : lmax + 1;
      jmin = min(jmin, lj[k]);
      lpc[k] = lmc[k] = lpp[k] = lmp[k] = f2{0.f, 0.f};
      scp[k] = scm[k] = 0;
  #pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (!SPIN) {
          double2 gn = make_double2(0, 0), gs = make_double2(0, 0);
          if (valid) {
            const double2 *gp = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
            gn = gp[0];
            if (pd.south) gs = gp[1];
          }
          g[k][j][0][0] = f2_of(gn.x + gs.x);
          g[k][j][0][1] = f2_of(gn.y + gs.y);
          g[k][j][1][0] = f2_of(gn.x - gs.x);
          g[k][j][1][1] = f2_of(gn.y - gs.y);
        } else {
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
          g[k][j][0][0] = f2_of(qn.x - un.y);
          g[k][j][0][1] = f2_of(qn.y + un.x);
          g[k][j][1][0] = f2_of(qn.x + un.y);
          g[k][j][1][1] = f2_of(qn.y - un.x);
          g[k][j][2][0] = f2_of(sg0 * (qs.x - us.y));
          g[k][j][2][1] = f2_of(sg0 * (qs.y + us.x));
          g[k][j][3][0] = f2_of(sg0 * (qs.x + us.y));
          g[k][j][3][1] = f2_of(sg0 * (qs.y - us.x));
        }
      }
    }

    // the tile starts at its pairs' earliest join block; the first tile of the group
    // zeroes the slot's degrees before it (the others leave their sums there)
    {
      const int wmin = __reduce_min_sync(0xffffffffu, jmin);
      if ((tid & 31) == 0) tstart[gi & 1][tid >> 5] = wmin;
    }
    __syncthreads();
    int lstart = tstart[gi & 1][0];
  #pragma unroll
    for (int w = 1; w < kAnaThreads / 32; ++w) lstart = min(lstart, tstart[gi & 1][w]);
    if (gi == 0)
      for (int i = tid; i < (min(lstart, lmax + 1) - l0) * V; i += kAnaThreads) outp[i] = 0.0;

    // one degree: this thread's V contributions (summed over its pairs) into c[];
    // the first term of each output is its exact product (no sum with zero)
    auto step = [&](int l, bool odd, bool act, f2 (&c)[V]) {
      // past lmax (second half of the last pair of degrees) the coefficients of
      // lmax stand in: the values are finite, never stored, and no table entry
      // outside this m is read
      const Coef32 cc = ld_coef32(cf + 2 * (l <= lmax ? l : lmax));
      const f2 nc = neg(cc.c);
  #pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const f2 wp = act ? lpc[k] : weight(lpc[k], scp[k]);
        if (!SPIN) {
  #pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const f2 gr = odd ? g[k][j][1][0] : g[k][j][0][0];
            const f2 gi = odd ? g[k][j][1][1] : g[k][j][0][1];
            if (k == 0) {
              c[2 * j] = mul(wp, gr);
              c[2 * j + 1] = mul(wp, gi);
            } else {
              acc_mul(c[2 * j], wp, gr.h, gr.l);
              acc_mul(c[2 * j + 1], wp, gi.h, gi.l);
            }
          }
          const f2 t = mul(cc.a, x[k]);
          const f2 ln = dot2(t, lpc[k], nc, lpp[k]);
          lpp[k] = lpc[k];
          lpc[k] = ln;
        } else {
          const f2 wm = act ? lmc[k] : weight(lmc[k], scm[k]);
          const f2 sp = odd ? neg(wp) : wp, sm = odd ? neg(wm) : wm;
  #pragma unroll
          for (int j = 0; j < NJ; ++j) {
            // T1 = W+_N l+ + (+-) W+_S l-,  T2 = W-_N l- + (+-) W-_S l+
            if (k == 0) {
              c[4 * j + 0] = mul(wp, g[k][j][0][0]);
              c[4 * j + 1] = mul(wp, g[k][j][0][1]);
              c[4 * j + 2] = mul(wm, g[k][j][1][0]);
              c[4 * j + 3] = mul(wm, g[k][j][1][1]);
            } else {
              acc_mul(c[4 * j + 0], wp, g[k][j][0][0].h, g[k][j][0][0].l);
              acc_mul(c[4 * j + 1], wp, g[k][j][0][1].h, g[k][j][0][1].l);
              acc_mul(c[4 * j + 2], wm, g[k][j][1][0].h, g[k][j][1][0].l);
              acc_mul(c[4 * j + 3], wm, g[k][j][1][1].h, g[k][j][1][1].l);
            }
            acc_mul(c[4 * j + 0], sm, g[k][j][2][0].h, g[k][j][2][0].l);
            acc_mul(c[4 * j + 1], sm, g[k][j][2][1].h, g[k][j][2][1].l);
            acc_mul(c[4 * j + 2], sp, g[k][j][3][0].h, g[k][j][3][0].l);
            acc_mul(c[4 * j + 3], sp, g[k][j][3][1].h, g[k][j][3][1].l);
          }
          const f2 t = mul(cc.a, x[k]);
          const f2 np_ = dot3(t, lpc[k], cc.ak, lpc[k], nc, lpp[k]);
          const f2 nm_ = dot3(t, lmc[k], neg(cc.ak), lmc[k], nc, lmp[k]);
          lpp[k] = lpc[k];
          lpc[k] = np_;
          lmp[k] = lmc[k];
          lmc[k] = nm_;
        }
      }
    };
    auto rescale_all = [&]() {
  #pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (scp[k] < 0 && fabsf(lpc[k].h) > kScaleUp32) {
          lpc[k] = {lpc[k].h * kScaleFactor32, lpc[k].l * kScaleFactor32};
          lpp[k] = {lpp[k].h * kScaleFactor32, lpp[k].l * kScaleFactor32};
          ++scp[k];
        }
        if (scm[k] < 0 && fabsf(lmc[k].h) > kScaleUp32) {
          lmc[k] = {lmc[k].h * kScaleFactor32, lmc[k].l * kScaleFactor32};
          lmp[k] = {lmp[k].h * kScaleFactor32, lmp[k].l * kScaleFactor32};
          ++scm[k];
        }
      }
    };
    auto put = [&](int q, const f2 (&c)[V]) {
  #pragma unroll
      for (int v = 0; v < V; ++v) slot[q * V + v][tid] = c[v];
    };

    auto recur = [&](int l) {  // recursion only
      const Coef32 cc = ld_coef32(cf + 2 * (l <= lmax ? l : lmax));
      const f2 nc = neg(cc.c);
  #pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const f2 t = mul(cc.a, x[k]);
        if (!SPIN) {
          const f2 ln = dot2(t, lpc[k], nc, lpp[k]);
          lpp[k] = lpc[k];
          lpc[k] = ln;
        } else {
          const f2 np_ = dot3(t, lpc[k], cc.ak, lpc[k], nc, lpp[k]);
          const f2 nm_ = dot3(t, lmc[k], neg(cc.ak), lmc[k], nc, lmp[k]);
          lpp[k] = lpc[k];
          lpc[k] = np_;
          lmp[k] = lmc[k];
          lmc[k] = nm_;
        }
      }
    };
    auto mode = [&]() {  // 0: all terms at scale 0, 2: all negligible, 1: weighted
      bool ok = true, dead = true;
  #pragma unroll
      for (int k = 0; k < PPT; ++k) {
        ok = ok && scp[k] == 0 && scm[k] == 0;
        dead = dead && negligible(lpc[k], scp[k]) && (!SPIN || negligible(lmc[k], scm[k]));
      }
      return __all_sync(0xffffffffu, ok) ? 0 : (__all_sync(0xffffffffu, dead) ? 2 : 1);
    };
    const f2 zero[V] = {};

    int since = 0;         // steps since the last exponent check
    bool settled = false;  // every lane's values at scale 0: they stay there (warp-uniform)
    int cb = 0;            // chunk parity: the quart buffer
    for (int lb = lstart; lb <= lmax; lb += LC) {
      // pairs joining at this degree take the recursion state where their terms start
      bool joins = false;
  #pragma unroll
      for (int k = 0; k < PPT; ++k)
        if (lj[k] == lb) {
          const int p = tile * (kAnaThreads * PPT) + tid + k * kAnaThreads;
          const JoinRec r = ld_join(a.join + ((size_t)mi * a.npairs + p) * 3);
          lpc[k] = r.lpc;
          lpp[k] = r.lpp;
          lmc[k] = r.lmc;
          lmp[k] = r.lmp;
          scp[k] = r.scp;
          scm[k] = r.scm;
          joins = true;
        }
      if (__any_sync(0xffffffffu, joins)) settled = false;
      // a warp none of whose lanes has joined holds zeros: it skips this chunk's
      // steps and adds zeros to the reduction
      const bool wlive = __any_sync(0xffffffffu, jmin <= lb);
      // this chunk's slot entry from the previous tiles (read early, added at the end)
      const bool mine = tid < 32 && lb + tid / V <= lmax;
      double *const o = outp + (int64_t)(lb - l0) * V + tid;
      const double prev = (gi > 0 && mine) ? *o : 0.0;
      if (!wlive) {
      } else if (LC >= 2) {
  #pragma unroll 1
        for (int q = 0; q < LC; q += 2) {
          const int l = lb + q;
          if (l > lmax) break;
          const int md = settled ? 0 : mode();
          settled = md == 0;
          if (md == 2) {
            recur(l);
            recur(l + 1);
            put(q, zero);
            put(q + 1, zero);
          } else {
            f2 c0[V], c1[V];
            if (md == 0) {
              step(l, false, true, c0);
              step(l + 1, true, true, c1);
            } else {
              step(l, false, false, c0);
              step(l + 1, true, false, c1);
            }
            put(q, c0);
            put(q + 1, c1);
          }
          since += 2;
          if (!settled && since >= 8) {
            rescale_all();
            since = 0;
          }
        }
      } else {  // one degree per chunk: parity alternates between chunks
        f2 c0[V];
        const bool odd = ((lb - l0) & 1) != 0;
        settled = settled || mode() == 0;
        if (settled) step(lb, odd, true, c0); else step(lb, odd, false, c0);
        put(0, c0);
        if (!settled && ++since >= 8) {
          rescale_all();
          since = 0;
        }
      }
      // a warp's slot columns are written and read by that warp only: warp-level sync
      __syncwarp();
      {  // 32 slots x kAnaThreads values: each warp sums its own 32 columns, then 4 partials per slot
        const int sl = tid & 31, part = tid >> 5;
        f2 t = {0.f, 0.f};
        if (wlive) {
          const f2 *row = &slot[sl][part * 32];
          t = row[0];
  #pragma unroll 8
          for (int i = 1; i < 32; ++i) t = f2_add_lazy(t, row[i]);
        }
        quart[cb][part][sl] = t;
      }
      __syncwarp();
      // one barrier per chunk: quart is double-buffered, so warp 0 reads this chunk's
      // partials while the others fill the other buffer, and it has read them before
      // it reaches the next barrier, after which this buffer is written again
      __syncthreads();
      if (tid < 32) {
        f2 t = quart[cb][0][tid];
  #pragma unroll
        for (int w = 1; w < kAnaThreads / 32; ++w) t = f2_add(t, quart[cb][w][tid]);
        if (mine) *o = prev + f2_val(t);
      }
      cb ^= 1;
    }
  }
}
// one-job shapes of up to two pairs a thread are held to 80 registers: six CTAs
// per SM instead of five (their shared slot table allows six); measured at one
// E/B pair, lmax 4095: 84.1 ms against 85.0 (two pairs) and 84.0 against 86.8 (one)
template <int NJ, int PPT, bool SPIN>
constexpr int mix_ana_min_blocks() {
  return (NJ == 1 && PPT <= 2) ? 6 : ((!SPIN && NJ == 1 && PPT == 4) ? 5 : 1);  // spin 0, 4 pairs: 96 registers
}
template <int NJ, int PPT, bool SPIN>
__global__ void __launch_bounds__(kAnaThreads, (mix_ana_min_blocks<NJ, PPT, SPIN>())) mix_ana(MixArgs a) {
  mix_ana_body<NJ, PPT, SPIN>(a, nullptr, a.ana_items[blockIdx.x]);
}
template <int NJ, int PPT, bool SPIN>
__global__ void __launch_bounds__(kAnaThreads, (mix_ana_min_blocks<NJ, PPT, SPIN>())) mix_ana_batch(const MixArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const MixArgs &a = args[it.w];
  mix_ana_body<NJ, PPT, SPIN>(a, tbl.p + a.ptr_off, make_int4(it.x, it.y, it.z, 0));
}

// ---------------------------------------------------------------------------
static MixArgs make_mix(const sht_plan_s *P, int polar) {
  MixArgs a;
  a.lmax = P->lmax;
  a.spin = P->spin;
  a.npairs = P->npairs;
  a.nm = P->nm;
  a.mval = P->d_mval;
  a.coef_off = P->d_coef_off;
  a.coef32 = P->d_coef32;
  a.alm32 = P->d_alm32;
  a.ncoef = P->ncoef;
  a.mpre = P->d_mpre;
  a.pairs = P->d_pairs;
  a.phase = P->d_phase;
  a.syn_items = P->d_syn_items[polar];
  a.ana_items = P->d_ana_items[polar];
  a.part_off = P->d_ana_part_off[polar];
  a.part = P->d_part;
  a.join = P->d_join;
  a.ptr_off = 0;
  return a;
}

// ---------------------------------------------------------------------------
// Join records (see JoinRec in mixed_common.cuh), once per plan: each thread runs
// its ring pair's recursion from l0 with the steps and rescale checks of the
// double-float kernels, records the state at every block of 16 degrees up to the
// first degree pair whose values are not negligible, then walks on to lmax + 1 for
// the bound on the values' true size.
// ---------------------------------------------------------------------------
template <bool SPIN>
__global__ void __launch_bounds__(128) join_kernel(MixArgs a, float4 *__restrict__ out, int min_exp) {
  const int mi = blockIdx.y, p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.npairs) return;
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax;
  const float4 *__restrict__ cf = a.coef32 + 2 * (a.coef_off[mi] - l0);
  const PairDev pd = a.pairs[p];
  const f3 x = f3_of(pd.x);
  f2 lpc, lmc = {0.f, 0.f}, lpp = {0.f, 0.f}, lmp = {0.f, 0.f};
  int scp, scm = 0;
  if (SPIN) {
    start_s(m, s, pd, a.mpre[mi], &lpc, &scp);
    start_s(m, -s, pd, a.mpre[mi], &lmc, &scm);
  } else {
    start_s0(m, pd, a.mpre[mi], &lpc, &scp);
  }
  // one recursion step at degree l (its row's coefficients; lmax's past lmax)
  auto step = [&](int l) {
    const Coef32 cc = ld_coef32(cf + 2 * (l <= lmax ? l : lmax));
    const f2 t = mul(cc.a, x);
    const f2 nc = neg(cc.c);
    if (SPIN) {
      const f2 np_ = dot3(t, lpc, cc.ak, lpc, nc, lpp);
      const f2 nm_ = dot3(t, lmc, neg(cc.ak), lmc, nc, lmp);
      lpp = lpc;
      lpc = np_;
      lmp = lmc;
      lmc = nm_;
    } else {
      const f2 ln = dot2(t, lpc, nc, lpp);
      lpp = lpc;
      lpc = ln;
    }
  };
  // the kernels' exponent check, made after every eight degrees from l0
  auto rescale = [&]() {
    if (scp < 0 && fabsf(lpc.h) > kScaleUp32) {
      lpc = {lpc.h * kScaleFactor32, lpc.l * kScaleFactor32};
      lpp = {lpp.h * kScaleFactor32, lpp.l * kScaleFactor32};
      ++scp;
    }
    if (SPIN && scm < 0 && fabsf(lmc.h) > kScaleUp32) {
      lmc = {lmc.h * kScaleFactor32, lmc.l * kScaleFactor32};
      lmp = {lmp.h * kScaleFactor32, lmp.l * kScaleFactor32};
      ++scm;
    }
  };
  JoinRec r = {lpc, lpp, lmc, lmp, scp, scm, l0, 0};
  bool live = false;
  int l = l0;
  for (; l <= lmax; l += 2) {
    const int off = l - l0;
    if (off % kJoinBlock == 0) r = {lpc, lpp, lmc, lmp, scp, scm, l, 0};
    if (!(negligible(lpc, scp) && (!SPIN || negligible(lmc, scm)))) {
      live = true;
      break;
    }
    step(l);
    step(l + 1);
    if ((off + 2) % 8 == 0) rescale();
  }
  // from the first live degree on: the largest true size (the kernels' weights:
  // scale 0 as is, scale -1 times 2^-104, below that dropped), low word included
  float vmax = 0.f;
  if (live) {
    auto size = [](f2 y, int sc) {
      const float v = fabsf(y.h) + fabsf(y.l);
      return sc == 0 ? v : (sc == -1 ? v * kScaleFactor32 : 0.f);
    };
    for (; l <= lmax + 1; ++l) {
      vmax = fmaxf(vmax, size(lpc, scp));
      if (SPIN) vmax = fmaxf(vmax, size(lmc, scm));
      if (l > lmax) break;
      step(l);
      if ((l + 1 - l0) % 8 == 0) rescale();
    }
  } else {
    r.lj = lmax + 1;
  }
  // 2^lexp >= vmax (with a margin of 2^-20 for the rounding of the bound), not
  // below 2^min_exp (the plan-wide bound / 2^16: finer grids would bring the
  // digit products near FP32's range end and add nothing)
  int e = min_exp;
  if (vmax > 0.f) {
    int ev;
    frexpf(vmax * (1.f + 0x1p-20f), &ev);  // vmax' = f 2^ev, f in [0.5, 1)
    e = max(e, ev);
  }
  r.lexp = e;
  float4 *o = out + ((size_t)mi * a.npairs + p) * 3;
  o[0] = make_float4(r.lpc.h, r.lpc.l, r.lpp.h, r.lpp.l);
  o[1] = make_float4(r.lmc.h, r.lmc.l, r.lmp.h, r.lmp.l);
  o[2] = make_float4(__int_as_float(r.scp), __int_as_float(r.scm), __int_as_float(r.lj), __int_as_float(r.lexp));
}

cudaError_t launch_join_records(const sht_plan_s *P, cudaStream_t st) {
  if (P->nm == 0 || P->npairs == 0) return cudaSuccess;
  const MixArgs a = make_mix(P, 1);
  const dim3 grid((P->npairs + 127) / 128, P->nm);
  int ub;
  frexpf(P->tc_lam_bound, &ub);  // tc_lam_bound = 2^(ub - 1)
  const int min_exp = ub - 1 - 16;
  if (P->spin) join_kernel<true><<<grid, 128, 0, st>>>(a, P->d_join, min_exp);
  else join_kernel<false><<<grid, 128, 0, st>>>(a, P->d_join, min_exp);
  return cudaGetLastError();
}

// Legendre stage over an explicit work list (stage 0: synthesis items int2, 1:
// analysis items int4); no a_lm conversion (launch_alm_prepare_mixed does it)
cudaError_t launch_leg_mixed_items(const sht_plan_s *P, int stage, int polar, const void *items, int n,
                                   cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  MixArgs a = make_mix(P, polar);
  const int nj = P->njobs_pad;
  if (stage == 0) {
    a.syn_items = static_cast<const int2 *>(items);
    if (P->tc_syn) return launch_leg_tc_syn(P, &a, n, st);
    if (P->spin == 0) {
      switch (nj) {
        case 1: mix_syn_s0<1><<<n, kSynTile, 0, st>>>(a); break;
        case 2: mix_syn_s0<2><<<n, kSynTile, 0, st>>>(a); break;
        case 4: mix_syn_s0<4><<<n, kSynTile, 0, st>>>(a); break;
        case 8: mix_syn_s0<8><<<n, kSynTile, 0, st>>>(a); break;
        default: mix_syn_s0<16><<<n, kSynTile, 0, st>>>(a); break;
      }
    } else {
      switch (nj) {
        case 1: mix_syn_spin<1><<<n, kSynTile, 0, st>>>(a); break;
        case 2: mix_syn_spin<2><<<n, kSynTile, 0, st>>>(a); break;
        case 4: mix_syn_spin<4><<<n, kSynTile, 0, st>>>(a); break;
        default: mix_syn_spin<8><<<n, kSynTile, 0, st>>>(a); break;
      }
    }
  } else {
    a.ana_items = static_cast<const int4 *>(items);
    if (P->tc_ana) return launch_leg_tc_ana(P, &a, n, st);
    if (P->spin == 0)
      ana_shape_s0(nj, P->ana_ppt, [&](auto sh) {
        mix_ana<decltype(sh)::nj, decltype(sh)::ppt, false><<<n, kAnaThreads, 0, st>>>(a);
      });
    else
      ana_shape_spin(nj, P->ana_ppt, [&](auto sh) {
        mix_ana<decltype(sh)::nj, decltype(sh)::ppt, true><<<n, kAnaThreads, 0, st>>>(a);
      });
  }
  return cudaGetLastError();
}

cudaError_t launch_leg_syn_mixed(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st, int mode) {
  cudaError_t e = launch_alm_prepare_mixed(P, alm, st, mode);
  if (e != cudaSuccess) return e;
  return launch_leg_mixed_items(P, 0, polar, P->d_syn_items[polar], P->nsyn_items[polar], st);
}

cudaError_t launch_leg_ana_mixed(const sht_plan_s *P, const DevPtrs &, int polar, cudaStream_t st) {
  return launch_leg_mixed_items(P, 1, polar, P->d_ana_items[polar], P->nana_items[polar], st);
}

}  // namespace sht

// ---------------------------------------------------------------------------
// batches (sht_batch_execute)
// ---------------------------------------------------------------------------
namespace sht {

size_t leg_mixed_args_size() { return sizeof(MixArgs); }

void leg_mixed_fill_args(const sht_plan_s *P, int polar, int ptr_off, void *out) {
  MixArgs a = make_mix(P, polar);
  a.ptr_off = ptr_off;
  memcpy(out, &a, sizeof(a));
}

cudaError_t launch_alm_prepare_mixed(const sht_plan_s *P, const DevPtrs &alm, cudaStream_t st, int mode) {
  if (P->nm == 0) return cudaSuccess;
  dim3 g(P->nm, P->spin ? P->njobs_pad : P->nmaps_pad);
  alm_to_f2<<<g, 256, 0, st>>>(P->lmax, P->spin, P->nm, P->nmaps_pad, P->astride, P->d_mval, P->d_mstart,
                               P->d_coef_off, P->ncoef, alm, P->d_alm32, mode);
  return cudaGetLastError();
}

cudaError_t launch_leg_mixed_batch(int stage, int spin, int nj, int ppt, const void *args, const int4 *items,
                                   int n, const PtrTable &tbl, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const MixArgs *a = static_cast<const MixArgs *>(args);
  if (stage == 0) {
    if (spin == 0) {
      switch (nj) {
        case 1: mix_syn_s0_batch<1><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 2: mix_syn_s0_batch<2><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 4: mix_syn_s0_batch<4><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 8: mix_syn_s0_batch<8><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        default: mix_syn_s0_batch<16><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
      }
    } else {
      switch (nj) {
        case 1: mix_syn_spin_batch<1><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 2: mix_syn_spin_batch<2><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        case 4: mix_syn_spin_batch<4><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
        default: mix_syn_spin_batch<8><<<n, kSynTile, 0, st>>>(a, items, tbl); break;
      }
    }
  } else {
    if (spin == 0)
      ana_shape_s0(nj, ppt, [&](auto sh) {
        mix_ana_batch<decltype(sh)::nj, decltype(sh)::ppt, false><<<n, kAnaThreads, 0, st>>>(a, items, tbl);
      });
    else
      ana_shape_spin(nj, ppt, [&](auto sh) {
        mix_ana_batch<decltype(sh)::nj, decltype(sh)::ppt, true><<<n, kAnaThreads, 0, st>>>(a, items, tbl);
      });
  }
  return cudaGetLastError();
}

}  // namespace sht
