// fft.cu -- ring FFTs of Eqs. syn1 and ana2.
//
// One CTA transforms one north/south ring pair of one map: the two real
// rings are packed as z = p_north + i p_south into a single complex DFT of
// length Nphi (pairs always share Nphi).  The ring lives in shared memory
// (up to kFftMaxLen points; longer rings in an L2-resident global scratch slot
// per CTA of a persistent grid) and is transformed in place: mixed-radix
// decimation-in-frequency passes (radix 2, 4 and small odd radices with each
// thread running whole butterflies, one barrier per pass; larger odd radices up
// to 127 as sweeps over the ring); the output comes out digit-reversed and is
// read back through a position table.  Lengths with a prime factor above
// 127 go through Rader's algorithm (prime n, n-1 smooth: a cyclic convolution
// of length n-1) or Bluestein's (chirp convolution of smooth length >= 2n-1);
// both convolutions run DIF forward and the transposed (DIT) passes back, so
// the result returns to natural order without a permutation pass.
//
// Synthesis, per ring:  p_x = sum_{m=-mmax}^{mmax} c_m e^{2 pi i m x / N},
//   c_m = F_m e^{i m phi0} (m >= 0), c_{-m} = conj(c_m); m is folded modulo N
//   when N <= 2 mmax (aliasing, Eq. syn1).
// Analysis, per ring:   G_m = w e^{-i m phi0} sum_x p_x e^{-2 pi i m x / N}  (Eq. ana2).
//
// The engine is written once over a number policy: IEEE double (F64, plans of
// the FP64 form) or double-float pairs on the FP32 pipe (DF, plans of the mixed
// form by default, see sht_plan_set_fft_precision: the FP32 pipe issues 64
// times the FP64 rate on GB300, and ~46 bits an operation keep the transform's
// relative error near 1e-14).  Ring pixels and the F_m / G_m arrays stay FP64 in
// memory; DF converts on the way in and out.  Phases e^{i m phi0} are walked
// along m (PhaseWalk) rather than evaluated per term.
#include <algorithm>
#include <mutex>
#include <set>
#include <vector>

#include "df.cuh"
#include "sht_internal.h"

namespace sht {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// cos(2 pi t / R) and sin(2 pi t / R) for odd radices R <= kMaxRadix, t = 1..(R-1)/2,
// in FP64 and as hi/lo float pairs, written once per device (fft_prepare_device).
// The butterflies index them with compile-time constants, so they are read as
// constant-bank operands.
__constant__ double c_cos[kMaxRadix + 1][kMaxRadix / 2 + 1];
__constant__ double c_sin[kMaxRadix + 1][kMaxRadix / 2 + 1];
__constant__ float2 c_cos2[kMaxRadix + 1][kMaxRadix / 2 + 1];
__constant__ float2 c_sin2[kMaxRadix + 1][kMaxRadix / 2 + 1];

// A complex double-float: re = (v.x, v.y), im = (v.z, v.w); 16 bytes like a
// double2 and moved as one 128-bit access.
struct cf2 {
  float4 v;
};

// Number policies.  C is the complex type the ring holds, S the type of its
// parts.  acc(s, x) adds x to a running sum and macc(s, x, c) adds x c (c real),
// both with the low word carried lazily in DF; fin() normalises such a sum.
// a_mi_b(A, B) = A - i B and a_pi_b(A, B) = A + i B.
struct F64 {
  using C = double2;
  using S = double;
  static constexpr int kRegRadix = kMaxRadix;  // largest odd radix with a register-resident butterfly
  static constexpr int kRollFrom = kMaxRadix + 2;  // odd radices whose outputs run one k at a time: none
  static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ C add(C a, C b) { return cadd(a, b); }
  static __device__ __forceinline__ C sub(C a, C b) { return csub(a, b); }
  static __device__ __forceinline__ C mul(C a, C b) { return cmul(a, b); }
  static __device__ __forceinline__ C conj(C a) { return cconj(a); }
  static __device__ __forceinline__ void acc(C &s, C x) { s = cadd(s, x); }
  static __device__ __forceinline__ void macc(C &s, C x, S c) {
    s.x = fma(x.x, c, s.x);
    s.y = fma(x.y, c, s.y);
  }
  static __device__ __forceinline__ void fin(C &) {}
  static __device__ __forceinline__ C a_mi_b(C A, C B) { return make_double2(A.x + B.y, A.y - B.x); }
  static __device__ __forceinline__ C a_pi_b(C A, C B) { return make_double2(A.x - B.y, A.y + B.x); }
  static __device__ __forceinline__ S re(C a) { return a.x; }
  static __device__ __forceinline__ S im(C a) { return a.y; }
  static __device__ __forceinline__ S sneg(S a) { return -a; }
  static __device__ __forceinline__ S kcos(int R, int t) { return c_cos[R][t]; }
  static __device__ __forceinline__ S ksin(int R, int t) { return c_sin[R][t]; }
  static __device__ __forceinline__ C ldg(const C *p) { return __ldg(p); }
  static __device__ __forceinline__ C of(double2 v) { return v; }
  static __device__ __forceinline__ double2 val(C v) { return v; }
  static __device__ __forceinline__ S scalar(double v) { return v; }
  static __device__ __forceinline__ C half(C a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
  static __device__ __forceinline__ C times_minus_i(C a) { return make_double2(a.y, -a.x); }
  static __device__ __forceinline__ C times_i(C a) { return make_double2(-a.y, a.x); }
  static __device__ __forceinline__ C scale(C a, S w) { return make_double2(a.x * w, a.y * w); }
  static __device__ __forceinline__ C scale2(C a, S wr, S wi) { return make_double2(a.x * wr, a.y * wi); }
  static __device__ __forceinline__ const C *tw(const FftPlanDev &fp) { return fp.w; }
  static __device__ __forceinline__ const C *spec(const FftPlanDev &fp) { return fp.spec; }
  static __device__ __forceinline__ const C *chirp(const FftPlanDev &fp) { return fp.chirp; }
};

struct DF {
  using C = cf2;
  using S = f2;
  static constexpr int kRegRadix = 13;  // above, the butterfly's pairs spill: sweeps instead
  // radices 11 and 13: the outputs one k at a time (the unrolled k loop spilled 76
  // bytes per thread at radix 13 under the 512-thread CTA's 128 registers)
  static constexpr int kRollFrom = 11;
  static __device__ __forceinline__ C mk(f2 r, f2 i) { return {make_float4(r.h, r.l, i.h, i.l)}; }
  static __device__ __forceinline__ S re(C a) { return {a.v.x, a.v.y}; }
  static __device__ __forceinline__ S im(C a) { return {a.v.z, a.v.w}; }
  static __device__ __forceinline__ C zero() { return {make_float4(0.f, 0.f, 0.f, 0.f)}; }
  static __device__ __forceinline__ C add(C a, C b) { return mk(f2_add(re(a), re(b)), f2_add(im(a), im(b))); }
  static __device__ __forceinline__ C sub(C a, C b) { return mk(f2_sub(re(a), re(b)), f2_sub(im(a), im(b))); }
  static __device__ __forceinline__ C mul(C a, C b) {
    return mk(dot2(re(a), re(b), neg(im(a)), im(b)), dot2(re(a), im(b), im(a), re(b)));
  }
  static __device__ __forceinline__ C conj(C a) { return {make_float4(a.v.x, a.v.y, -a.v.z, -a.v.w)}; }
  static __device__ __forceinline__ void acc(C &s, C x) {
    s = mk(f2_add_lazy(re(s), re(x)), f2_add_lazy(im(s), im(x)));
  }
  static __device__ __forceinline__ f2 madd(f2 s, f2 x, f2 c) {
    const f2 p = sht::mul(x, c);
    const f2 t = two_sum(s.h, p.h);
    return {t.h, __fadd_rn(s.l, __fadd_rn(t.l, p.l))};
  }
  static __device__ __forceinline__ void macc(C &s, C x, S c) { s = mk(madd(re(s), re(x), c), madd(im(s), im(x), c)); }
  static __device__ __forceinline__ void fin(C &s) {
    s = mk(fast_two_sum(s.v.x, s.v.y), fast_two_sum(s.v.z, s.v.w));
  }
  static __device__ __forceinline__ C a_mi_b(C A, C B) { return mk(f2_add(re(A), im(B)), f2_sub(im(A), re(B))); }
  static __device__ __forceinline__ C a_pi_b(C A, C B) { return mk(f2_sub(re(A), im(B)), f2_add(im(A), re(B))); }
  static __device__ __forceinline__ S sneg(S a) { return neg(a); }
  static __device__ __forceinline__ S kcos(int R, int t) {
    const float2 c = c_cos2[R][t];
    return {c.x, c.y};
  }
  static __device__ __forceinline__ S ksin(int R, int t) {
    const float2 c = c_sin2[R][t];
    return {c.x, c.y};
  }
  static __device__ __forceinline__ C ldg(const C *p) { return {__ldg(&p->v)}; }
  static __device__ __forceinline__ C of(double2 v) { return mk(f2_split(v.x), f2_split(v.y)); }
  static __device__ __forceinline__ double2 val(C a) { return make_double2(f2_join(re(a)), f2_join(im(a))); }
  static __device__ __forceinline__ S scalar(double v) { return f2_of(v); }
  static __device__ __forceinline__ C half(C a) {  // exact (outside FP32's subnormal range)
    return {make_float4(0.5f * a.v.x, 0.5f * a.v.y, 0.5f * a.v.z, 0.5f * a.v.w)};
  }
  static __device__ __forceinline__ C times_minus_i(C a) { return {make_float4(a.v.z, a.v.w, -a.v.x, -a.v.y)}; }
  static __device__ __forceinline__ C times_i(C a) { return {make_float4(-a.v.z, -a.v.w, a.v.x, a.v.y)}; }
  static __device__ __forceinline__ C scale(C a, S w) { return scale2(a, w, w); }
  static __device__ __forceinline__ C scale2(C a, S wr, S wi) {  // real part times wr, imaginary part times wi
    const f2 r = sht::mul(re(a), wr), i = sht::mul(im(a), wi);
    return mk(fast_two_sum(r.h, r.l), fast_two_sum(i.h, i.l));
  }
  static __device__ __forceinline__ const C *tw(const FftPlanDev &fp) { return reinterpret_cast<const C *>(fp.wf); }
  static __device__ __forceinline__ const C *spec(const FftPlanDev &fp) {
    return reinterpret_cast<const C *>(fp.specf);
  }
  static __device__ __forceinline__ const C *chirp(const FftPlanDev &fp) {
    return reinterpret_cast<const C *>(fp.chirpf);
  }
};

// y_s = sum_r x_r e^{-2 pi i r s / R} for s < R; out(s, y_s) receives each output.
// Odd R uses the symmetric form: with S_j = x_j + x_{R-j}, D_j = x_j - x_{R-j},
//   y_k = A_k - i B_k,  y_{R-k} = A_k + i B_k,
//   A_k = x_0 + sum_j S_j cos(2 pi j k / R),  B_k = sum_j D_j sin(2 pi j k / R),
// i.e. 4 h^2 real multiply-adds for R points (h = (R-1)/2) instead of 4 R^2.
template <int R, class N, class Out>
__device__ __forceinline__ void dft_small(typename N::C (&x)[R], Out &&out) {
  using C = typename N::C;
  using S = typename N::S;
  if constexpr (R == 2) {
    out(0, N::add(x[0], x[1]));
    out(1, N::sub(x[0], x[1]));
  } else if constexpr (R == 4) {
    const C s02 = N::add(x[0], x[2]), d02 = N::sub(x[0], x[2]);
    const C s13 = N::add(x[1], x[3]), d13 = N::sub(x[1], x[3]);
    out(0, N::add(s02, s13));
    out(1, N::a_mi_b(d02, d13));
    out(2, N::sub(s02, s13));
    out(3, N::a_pi_b(d02, d13));
  } else {
    static_assert(R % 2 == 1 && R <= kMaxRadix, "odd radix");
    constexpr int h = (R - 1) / 2;
    const C x0 = x[0];
    C y0 = x0;
#pragma unroll
    for (int j = 1; j <= h; ++j) {  // S_j into x[j], D_j into x[R-j]
      const C a = x[j], b = x[R - j];
      x[j] = N::add(a, b);
      x[R - j] = N::sub(a, b);
      N::acc(y0, x[j]);
    }
    N::fin(y0);
    out(0, y0);
    // (N::kRollFrom: from that radix on the outputs run one k at a time, so that not
    // every k's constants and accumulators are live at once)
#pragma unroll(R >= N::kRollFrom ? 1 : h)
    for (int k = 1; k <= h; ++k) {
      C A = x0, B = N::zero();
#pragma unroll
      for (int j = 1; j <= h; ++j) {
        const int t = (j * k) % R;
        const S c = N::kcos(R, t <= h ? t : R - t);
        const S sn = t <= h ? N::ksin(R, t) : N::sneg(N::ksin(R, R - t));
        N::macc(A, x[j], c);
        N::macc(B, x[R - j], sn);
      }
      N::fin(A);
      N::fin(B);
      out(k, N::a_mi_b(A, B));
      out(R - k, N::a_pi_b(A, B));
    }
  }
}

// The ring buffer: the kernels' dynamic shared memory, named at namespace scope
// so the out-of-line passes address it as shared memory.
extern __shared__ double2 s_ring[];

// Where a ring of element type C lives while it is transformed: shared memory
// (every length up to kFftMaxLen), or a CTA-private slot of global scratch for
// longer rings, which stays in L2 (the engine is the same; barriers order global
// accesses within the CTA as they do shared ones).
template <class C>
struct SharedRing {
  __device__ __forceinline__ C *at(int i) const { return reinterpret_cast<C *>(s_ring) + i; }
};
template <class C>
struct GlobalRing {
  C *p;
  __device__ __forceinline__ C *at(int i) const { return p + i; }
};

// One in-place pass of radix R over the len / L blocks of length L of the ring.
// Butterfly (block B, offset b < L/R) works on ring[B L + b + r L/R], r < R:
//   decimation in frequency (DIT = false): DFT_R, then output s times W_L^{s b};
//   its transpose (DIT = true): input r times W_L^{r b}, then DFT_R.
// Each butterfly touches only its own R slots, so one barrier per pass suffices.
// W holds e^{-2 pi i k / len}; W_L^e = W[e len / L].
template <int R, bool DIT, class N, class Ring>
__device__ __noinline__ void fft_stage(Ring ring, int len, int L, const typename N::C *__restrict__ W) {
  using C = typename N::C;
  const int LR = L / R;
  const int nb = len / R;
  const int tw = len / L;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) {
    const int B = q / LR, b = q - B * LR;
    C *p = ring.at(B * L + b);
    C x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = p[r * LR];
    if (DIT && b != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = N::mul(x[r], N::ldg(W + r * b * tw));
    }
    dft_small<R, N>(x, [&](int s, C y) {
      if (!DIT && s != 0 && b != 0) y = N::mul(y, N::ldg(W + s * b * tw));
      p[s * LR] = y;
    });
  }
  __syncthreads();
}

// One in-place pass of an odd radix R in (N::kRegRadix, kMaxBigRadix], the same
// butterflies as fft_stage.  R values no longer fit in one thread's registers, so
// the symmetric form of dft_small runs as sweeps over the ring:
//   1. S_j = x_j + x_{R-j} into slot j and D_j = x_j - x_{R-j} into slot R-j
//      (j = 1..h, after the input twiddles for DIT), one item per (butterfly, j);
//   2. in rounds of whole butterflies, one item per (butterfly, k), k = 0..h,
//      computes y_k and y_{R-k} from x_0, S and D into registers; after a barrier
//      the items write them back in place (DIF: times the output twiddles).
// Items are k-major so that a warp shares k (its cos/sin loads broadcast) and
// walks consecutive butterflies (consecutive slots).  cos and sin of 2 pi t / R
// come from the ring's own table: W[t len / R] = e^{-2 pi i t / R}.  The DF
// sums are normalised every 8 terms.
template <bool DIT, class N, class Ring>
__device__ __noinline__ void fft_stage_big(Ring ring, int len, int L, int R, const typename N::C *__restrict__ W) {
  using C = typename N::C;
  constexpr int kItems = 4;  // output pairs a thread holds across the barrier
  const int LR = L / R, nb = len / R, tw = len / L, h = (R - 1) / 2, tr = len / R;
  for (int i = threadIdx.x; i < nb * h; i += blockDim.x) {
    const int j = 1 + i / nb, q = i % nb;
    const int B = q / LR, b = q - B * LR;
    C *p = ring.at(B * L + b);
    C u = p[j * LR], v = p[(R - j) * LR];
    if (DIT && b != 0) {
      u = N::mul(u, N::ldg(W + j * b * tw));
      v = N::mul(v, N::ldg(W + (R - j) * b * tw));
    }
    p[j * LR] = N::add(u, v);
    p[(R - j) * LR] = N::sub(u, v);
  }
  __syncthreads();
  const int per = h + 1;
  int nround = (int)(blockDim.x * kItems) / per;  // butterflies per round
  if (nround >= 32) nround &= ~31;
  for (int q0 = 0; q0 < nb; q0 += nround) {
    const int nq = min(nround, nb - q0), nit = nq * per;
    C ya[kItems], yb[kItems];
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int i = threadIdx.x + u * blockDim.x;
      if (i < nit) {
        const int k = i / nq, q = q0 + i % nq;
        const int B = q / LR, b = q - B * LR;
        const C *p = ring.at(B * L + b);
        C A = p[0];
        if (k == 0) {
          for (int j = 1; j <= h; ++j) {
            N::acc(A, p[j * LR]);
            if ((j & 7) == 0) N::fin(A);
          }
          N::fin(A);
          ya[u] = A;
        } else {
          C Bn = N::zero();  // -(sum_j D_j sin(2 pi j k / R))
          int t = 0;
          for (int j = 1; j <= h; ++j) {
            t += k;
            if (t >= R) t -= R;
            const C w = N::ldg(W + t * tr);
            N::macc(A, p[j * LR], N::re(w));
            N::macc(Bn, p[(R - j) * LR], N::im(w));
            if ((j & 7) == 0) {
              N::fin(A);
              N::fin(Bn);
            }
          }
          N::fin(A);
          N::fin(Bn);
          ya[u] = N::a_pi_b(A, Bn);  // y_k = A - i B
          yb[u] = N::a_mi_b(A, Bn);  // y_{R-k} = A + i B
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int i = threadIdx.x + u * blockDim.x;
      if (i < nit) {
        const int k = i / nq, q = q0 + i % nq;
        const int B = q / LR, b = q - B * LR;
        C *p = ring.at(B * L + b);
        C y0 = ya[u];
        if (k == 0) {
          p[0] = y0;
        } else {
          C y1 = yb[u];
          if (!DIT && b != 0) {
            y0 = N::mul(y0, N::ldg(W + k * b * tw));
            y1 = N::mul(y1, N::ldg(W + (R - k) * b * tw));
          }
          p[k * LR] = y0;
          p[(R - k) * LR] = y1;
        }
      }
    }
    __syncthreads();
  }
}

// radix R with its butterflies in registers up to N::kRegRadix, else as sweeps
template <int R, bool DIT, class N, class Ring>
__device__ __forceinline__ void fft_stage_r(Ring ring, int len, int L, const typename N::C *W) {
  if constexpr (R <= N::kRegRadix)
    fft_stage<R, DIT, N>(ring, len, L, W);
  else
    fft_stage_big<DIT, N>(ring, len, L, R, W);
}

template <bool DIT, class N, class Ring>
__device__ void fft_stage_any(Ring ring, int len, int L, int R, const typename N::C *W) {
  switch (R) {
    case 2: fft_stage<2, DIT, N>(ring, len, L, W); break;
    case 3: fft_stage<3, DIT, N>(ring, len, L, W); break;
    case 4: fft_stage<4, DIT, N>(ring, len, L, W); break;
    case 5: fft_stage<5, DIT, N>(ring, len, L, W); break;
    case 7: fft_stage<7, DIT, N>(ring, len, L, W); break;
    case 11: fft_stage_r<11, DIT, N>(ring, len, L, W); break;
    case 13: fft_stage_r<13, DIT, N>(ring, len, L, W); break;
    case 17: fft_stage_r<17, DIT, N>(ring, len, L, W); break;
    case 19: fft_stage_r<19, DIT, N>(ring, len, L, W); break;
    case 23: fft_stage_r<23, DIT, N>(ring, len, L, W); break;
    case 29: fft_stage_r<29, DIT, N>(ring, len, L, W); break;
    case 31: fft_stage_r<31, DIT, N>(ring, len, L, W); break;
    default: fft_stage_big<DIT, N>(ring, len, L, R, W); break;
  }
}

// Forward DFT of ring[0..fp.len) by decimation in frequency: natural-order input,
// output X_k at position fp.pos[k] (mixed-radix digit reversal).
template <class N, class Ring>
__device__ void fft_dif(Ring ring, const FftPlanDev &fp) {
  int L = fp.len;
  for (int i = 0; i < fp.nrad; ++i) {
    fft_stage_any<false, N>(ring, fp.len, L, fp.rad[i], N::tw(fp));
    L /= fp.rad[i];
  }
}

// The transpose of fft_dif (its passes transposed, in reverse order): input
// z_k at position fp.pos[k], output the forward DFT of z in natural order.
template <class N, class Ring>
__device__ void fft_dit(Ring ring, const FftPlanDev &fp) {
  int L = 1;
  for (int i = fp.nrad - 1; i >= 0; --i) {
    L *= fp.rad[i];
    fft_stage_any<true, N>(ring, fp.len, L, fp.rad[i], N::tw(fp));
  }
}

// Full forward DFT of length n of the data placed by the caller:
//   kind 0: buf[k] = x_k (k < n);
//   kind 1: buf[q] = x_{g^q} (q < n-1), *x0 = x_0;
//   kind 2: buf[k] = x_k chirp_k (k < n), 0 up to len.
// Afterwards dft_at(k) returns X_k.  Kinds 1 and 2 are cyclic convolutions with
// a kernel whose spectrum was made by fft_dif (so it is digit-reversed like the
// data): DIF, pointwise product, then the inverse as conj(DIT(conj)), which
// returns to natural order with no permutation pass.
template <class N, class Ring>
__device__ void dft_run(Ring ring, const FftPlanDev &fp, typename N::C *sh_x0, typename N::C *sh_a0) {
  typename N::C *const buf = ring.at(0);
  fft_dif<N>(ring, fp);
  if (fp.kind == 0) return;
  if (fp.kind == 1 && threadIdx.x == 0) *sh_a0 = buf[0];  // X_0 sits at position 0
  __syncthreads();
  const typename N::C *spec = N::spec(fp);
  for (int i = threadIdx.x; i < fp.len; i += blockDim.x) buf[i] = N::conj(N::mul(buf[i], N::ldg(spec + i)));
  __syncthreads();
  fft_dit<N>(ring, fp);
}

template <class N>
__device__ __forceinline__ typename N::C dft_at(const typename N::C *buf, const FftPlanDev &fp, int k,
                                                typename N::C x0, typename N::C a0) {
  if (fp.kind == 0) return buf[__ldg(fp.pos + k)];
  if (fp.kind == 1) {
    if (k == 0) return N::add(x0, a0);
    return N::add(x0, N::conj(buf[fp.inv_out[k]]));
  }
  return N::mul(N::ldg(N::chirp(fp) + k), N::conj(buf[k]));
}

// ---------------------------------------------------------------------------
// spectrum precomputation (plan time, FP64): dst = scale * DFT_len(src)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFftThreads) spectrum_kernel(const FftPlanDev *fpd, const double2 *src,
                                                              double2 *dst, int len, double scale) {
  double2 *const buf = s_ring;
  const FftPlanDev fp = *fpd;
  for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = src[i];
  __syncthreads();
  fft_dif<F64>(SharedRing<double2>{}, fp);
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = make_double2(buf[i].x * scale, buf[i].y * scale);
}
// the same for lengths beyond shared memory: transformed in place in dst
__global__ void __launch_bounds__(kFftThreads) spectrum_kernel_global(const FftPlanDev *fpd, const double2 *src,
                                                                     double2 *dst, int len, double scale) {
  const FftPlanDev fp = *fpd;
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  fft_dif<F64>(GlobalRing<double2>{dst}, fp);
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = make_double2(dst[i].x * scale, dst[i].y * scale);
}

cudaError_t launch_fft_spectrum(const FftPlanDev *hp, const FftPlanDev *dp, const double2 *src, double2 *dst,
                                int len, double scale, cudaStream_t st) {
  if (len > kFftMaxLen) {
    spectrum_kernel_global<<<1, kFftThreads, 0, st>>>(dp, src, dst, len, scale);
  } else {
    const int smem = len * (int)sizeof(double2);  // limit raised by fft_prepare_device
    spectrum_kernel<<<1, kFftThreads, smem, st>>>(dp, src, dst, len, scale);
  }
  return cudaGetLastError();
}

// e^{i m phi0} with the product m*phi0 carried to ~1e-32 before the sincos.
// Callers skip rings with phi0 = 0; out of line so that no part of the sincos
// (its FP64 range tests) is predicated into their loops for every coefficient.
__device__ __noinline__ double2 phase_of(int m, double phi0) {
  if (m == 0) return make_double2(1.0, 0.0);
  const double dm = (double)m;
  const double hi = dm * phi0;
  const double lo = fma(dm, phi0, -hi);
  double s, c;
  sincos(hi, &s, &c);
  return make_double2(c - s * lo, s + c * lo);
}

struct FftArgs {
  int nm, npairs, mmax;
  const int *mval;
  const int *minv;
  const int *syn_first;
  const int2 *pair_rings;
  const RingDev *rings;
  const FftPlanDev *plans;
  const int *pair_fft;
  double2 *phase;
  DevPtrs map;
  int weighted, add;
  int ptr_off;
  int nmaps_run;  // maps per side (global-ring kernels walk npairs_run x nmaps_run items)
  int pair0, npairs_run;  // the ring pairs [pair0, pair0 + npairs_run) one launch transforms
  int m_identity;         // mval[mi] = mi for every mi (the phases can be walked along m)
};

// ---------------------------------------------------------------------------
// synthesis: F (per m) -> ring pixels
// ---------------------------------------------------------------------------
// e^{i m phi} for m = m0, m0 + step, m0 + 2 step, ... in the engine's arithmetic:
// one sincos for the first value and one for the step, then one product a step
// (its rounding adds up over at most a ring's length / blockDim steps)
template <class N>
struct PhaseWalk {
  typename N::C e, s;
  __device__ __forceinline__ void init(int m0, int step, double phi) {
    e = N::of(phase_of(m0, phi));
    s = N::of(phase_of(step, phi));
  }
  __device__ __forceinline__ void next() { e = N::mul(e, s); }
};

// The term of coefficient m for one ring pair, conj?(cN e^{i m phiN}) + i conj?(cS e^{i m phiS})
// (conj_ for the m < 0 half of the sum), in the engine's arithmetic; pn, ps are the
// phases e^{i m phi} of rings with phi0 != 0 (ph_n, ph_s).  F below the first pair
// the Legendre stage processed for this m is zero.
template <class N>
__device__ __forceinline__ typename N::C synth_term(const FftArgs &a, int j, int p, int m, bool south, bool conj_,
                                                    bool ph_n, bool ph_s, typename N::C pn, typename N::C ps) {
  using C = typename N::C;
  const int mi = a.minv[m];
  if (mi < 0 || p < a.syn_first[mi]) return N::zero();
  const double2 *f = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
  C z = N::of(f[0]);
  if (ph_n) z = N::mul(z, pn);
  if (conj_) z = N::conj(z);
  if (south) {
    C zs = N::of(f[1]);
    if (ph_s) zs = N::mul(zs, ps);
    if (conj_) zs = N::conj(zs);
    z = N::add(z, N::times_i(zs));
  }
  return z;
}

// Z_k = sum_{m >= 0, m = k mod N} (cN_m + i cS_m) + sum_{m >= 1, -m = k mod N} (conj cN_m + i conj cS_m),
// c_m = F_m e^{i m phi0}.  The first term starts the sum (without aliasing, N > 2 mmax,
// it is the only one).  en, es = e^{i k phi}, bn, bs = e^{i N phi} of the two rings:
// the term m = k + N i has phase e^{i k phi} (e^{i N phi})^i, the conjugate term
// m = N (i + 1) - k has e^{-i k phi} (e^{i N phi})^(i + 1).
template <class N>
__device__ typename N::C spectrum_at(const FftArgs &a, int j, int p, int k, int Nr, bool south, bool ph_n, bool ph_s,
                                     typename N::C en, typename N::C es, typename N::C bn, typename N::C bs) {
  using C = typename N::C;
  const int mc = k == 0 ? Nr : Nr - k;  // first m of the conjugate terms
  C z = N::zero();
  bool first = true;
  auto add = [&](int m, bool cj, C pn, C ps) {
    const C t = synth_term<N>(a, j, p, m, south, cj, ph_n, ph_s, pn, ps);
    z = first ? t : N::add(z, t);
    first = false;
  };
  C pn = en, ps = es;
  for (int m = k; m <= a.mmax; m += Nr) {
    add(m, false, pn, ps);
    if (ph_n) pn = N::mul(pn, bn);
    if (ph_s) ps = N::mul(ps, bs);
  }
  if (mc <= a.mmax) {
    C qn = N::conj(en), qs = N::conj(es);
    if (ph_n) qn = N::mul(qn, bn);
    if (ph_s) qs = N::mul(qs, bs);
    for (int m = mc; m <= a.mmax; m += Nr) {
      add(m, true, qn, qs);
      if (ph_n) qn = N::mul(qn, bn);
      if (ph_s) qs = N::mul(qs, bs);
    }
  }
  return z;
}

template <class N, class Ring>
__device__ __forceinline__ void fft_syn_kernel_body(Ring ring, const FftArgs &a, double *const *ptrs, const int p,
                                     const int j) {
  using C = typename N::C;
  C *const buf = ring.at(0);
  __shared__ C sh_x0, sh_a0;
  const FftPlanDev fp = a.plans[a.pair_fft[p]];
  const int2 rr = a.pair_rings[p];
  const RingDev rn = a.rings[rr.x];
  const bool south = rr.y >= 0;
  const RingDev rs = a.rings[south ? rr.y : rr.x];
  const int Nphi = fp.n;
  const bool ph_n = rn.phi0 != 0.0, ph_s = south && rs.phi0 != 0.0;
  // the spectrum in natural order k = tid, tid + blockDim, ..., with the rings'
  // phases walked along; inverse DFT via conj(DFT(conj(Z))).  Rader's input order
  // is q with g^q = k: q = (N-1 - inv_out[k]) mod (N-1), as g^{-inv_out[k]} = k.
  PhaseWalk<N> phn, phs;
  C bn = N::zero(), bs = N::zero();
  if (ph_n) {
    phn.init(threadIdx.x, blockDim.x, rn.phi0);
    bn = N::of(phase_of(Nphi, rn.phi0));
  }
  if (ph_s) {
    phs.init(threadIdx.x, blockDim.x, rs.phi0);
    bs = N::of(phase_of(Nphi, rs.phi0));
  }
  const C *chirp = N::chirp(fp);
  for (int k = threadIdx.x; k < Nphi; k += blockDim.x) {
    const C z = N::conj(spectrum_at<N>(a, j, p, k, Nphi, south, ph_n, ph_s, phn.e, phs.e, bn, bs));
    if (fp.kind == 0) {
      buf[k] = z;
    } else if (fp.kind == 1) {
      if (k == 0)
        sh_x0 = z;
      else
        buf[(Nphi - 1 - fp.inv_out[k]) % (Nphi - 1)] = z;
    } else {
      buf[k] = N::mul(z, N::ldg(chirp + k));
    }
    if (ph_n) phn.next();
    if (ph_s) phs.next();
  }
  if (fp.kind == 2)
    for (int k = Nphi + threadIdx.x; k < fp.len; k += blockDim.x) buf[k] = N::zero();
  __syncthreads();
  dft_run<N>(ring, fp, &sh_x0, &sh_a0);
  const C x0 = sh_x0, a0 = sh_a0;
  double *mp = ptrs[j];
  const int weighted = a.weighted;
  const typename N::S wn = N::scalar(rn.weight), ws = N::scalar(rs.weight);
  for (int x = threadIdx.x; x < Nphi; x += blockDim.x) {
    C zc = N::conj(dft_at<N>(buf, fp, x, x0, a0));  // north = Re z, south = Im z
    if (weighted) zc = N::scale2(zc, wn, ws);
    const double2 z = N::val(zc);
    double vn = z.x;
    double *on = mp + rn.ofs + (int64_t)x * rn.stride;
    if (a.add) vn += *on;
    *on = vn;
    if (south) {
      double vs = z.y;
      double *os = mp + rs.ofs + (int64_t)x * rs.stride;
      if (a.add) vs += *os;
      *os = vs;
    }
  }
}
template <class N>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_syn_kernel(FftArgs a) {
  fft_syn_kernel_body<N>(SharedRing<typename N::C>{}, a, a.map.p, a.pair0 + blockIdx.x, blockIdx.y);
}
template <class N>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_syn_kernel_batch(const FftArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const FftArgs &a = args[it.w];
  fft_syn_kernel_body<N>(SharedRing<typename N::C>{}, a, tbl.p + a.ptr_off, it.x, it.y);
}

// ---------------------------------------------------------------------------
// analysis: ring pixels -> G (per m)
// ---------------------------------------------------------------------------
template <class N, class Ring>
__device__ __forceinline__ void fft_ana_kernel_body(Ring ring, const FftArgs &a, double *const *ptrs, const int p,
                                     const int j) {
  using C = typename N::C;
  C *const buf = ring.at(0);
  __shared__ C sh_x0, sh_a0;
  const FftPlanDev fp = a.plans[a.pair_fft[p]];
  const int2 rr = a.pair_rings[p];
  const RingDev rn = a.rings[rr.x];
  const bool south = rr.y >= 0;
  const RingDev rs = a.rings[south ? rr.y : rr.x];
  const int Nphi = fp.n;
  const double *mp = ptrs[j];
  auto zin = [&](int x) {
    const double vn = mp[rn.ofs + (int64_t)x * rn.stride];
    const double vs = south ? mp[rs.ofs + (int64_t)x * rs.stride] : 0.0;
    return make_double2(vn, vs);
  };
  if (fp.kind == 0) {
    for (int k = threadIdx.x; k < Nphi; k += blockDim.x) buf[k] = N::of(zin(k));
  } else if (fp.kind == 1) {
    for (int q = threadIdx.x; q < Nphi - 1; q += blockDim.x) buf[q] = N::of(zin(fp.perm_in[q]));
    if (threadIdx.x == 0) sh_x0 = N::of(zin(0));
  } else {
    const C *chirp = N::chirp(fp);
    for (int k = threadIdx.x; k < fp.len; k += blockDim.x)
      buf[k] = (k < Nphi) ? N::mul(N::of(zin(k)), N::ldg(chirp + k)) : N::zero();
  }
  __syncthreads();
  dft_run<N>(ring, fp, &sh_x0, &sh_a0);
  const C x0 = sh_x0, a0 = sh_a0;
  const int weighted = a.weighted;
  const typename N::S wn = N::scalar(rn.weight), ws = N::scalar(rs.weight);
  const bool ph_n = rn.phi0 != 0.0, ph_s = south && rs.phi0 != 0.0;
  // phases e^{i m phi}: walked along m = mi when the m list is 0, 1, 2, ...
  const bool walk = a.m_identity;
  PhaseWalk<N> wpn, wps;
  if (ph_n && walk) wpn.init(threadIdx.x, blockDim.x, rn.phi0);
  if (ph_s && walk) wps.init(threadIdx.x, blockDim.x, rs.phi0);
  for (int mi = threadIdx.x; mi < a.nm; mi += blockDim.x) {
    const int m = a.mval[mi];
    const int k = m % Nphi, kn = (Nphi - k) % Nphi;
    const C Zk = dft_at<N>(buf, fp, k, x0, a0), Zn = N::conj(dft_at<N>(buf, fp, kn, x0, a0));
    // P_N = (Zk + conj Zn)/2,  P_S = (Zk - conj Zn)/(2i), in the engine's arithmetic
    C pn = N::half(N::add(Zk, Zn)), ps = N::half(N::times_minus_i(N::sub(Zk, Zn)));
    if (weighted) {
      pn = N::scale(pn, wn);
      ps = N::scale(ps, ws);
    }
    if (ph_n) {
      pn = N::mul(pn, N::conj(walk ? wpn.e : N::of(phase_of(m, rn.phi0))));
      if (walk) wpn.next();
    }
    if (ph_s) {
      ps = N::mul(ps, N::conj(walk ? wps.e : N::of(phase_of(m, rs.phi0))));
      if (walk) wps.next();
    }
    const double2 gn = N::val(pn);
    const double2 gs = south ? N::val(ps) : make_double2(0.0, 0.0);
    double2 *g = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
    g[0] = gn;
    g[1] = gs;
  }
}
template <class N>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_ana_kernel(FftArgs a) {
  fft_ana_kernel_body<N>(SharedRing<typename N::C>{}, a, a.map.p, a.pair0 + blockIdx.x, blockIdx.y);
}
template <class N>
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_ana_kernel_batch(const FftArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const FftArgs &a = args[it.w];
  fft_ana_kernel_body<N>(SharedRing<typename N::C>{}, a, tbl.p + a.ptr_off, it.x, it.y);
}

// Rings longer than shared memory holds: a persistent grid, each CTA owning one
// scratch slot of slot_len points, walks the (pair, map) items in turn.
template <class N>
__global__ void __launch_bounds__(kFftThreads) fft_syn_kernel_global(FftArgs a, double2 *scratch,
                                                                     int slot_len) {
  using C = typename N::C;
  const GlobalRing<C> ring{reinterpret_cast<C *>(scratch + (size_t)blockIdx.x * slot_len)};
  const int n = a.npairs_run * a.nmaps_run;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    fft_syn_kernel_body<N>(ring, a, a.map.p, a.pair0 + it % a.npairs_run, it / a.npairs_run);
    __syncthreads();  // the slot is rewritten by the next item
  }
}
template <class N>
__global__ void __launch_bounds__(kFftThreads) fft_ana_kernel_global(FftArgs a, double2 *scratch,
                                                                     int slot_len) {
  using C = typename N::C;
  const GlobalRing<C> ring{reinterpret_cast<C *>(scratch + (size_t)blockIdx.x * slot_len)};
  const int n = a.npairs_run * a.nmaps_run;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    fft_ana_kernel_body<N>(ring, a, a.map.p, a.pair0 + it % a.npairs_run, it / a.npairs_run);
    __syncthreads();
  }
}

static FftArgs make_fft_args(const sht_plan_s *P, const DevPtrs &map, int polar) {
  FftArgs a;
  a.nm = P->nm;
  a.npairs = P->npairs;
  a.mmax = P->mmax;
  a.mval = P->d_mval;
  a.minv = P->d_minv;
  a.syn_first = P->d_syn_first[polar];
  a.pair_rings = P->d_pair_rings;
  a.rings = P->d_rings;
  a.plans = P->d_fft;
  a.pair_fft = P->d_pair_fft;
  a.phase = P->d_phase;
  a.map = map;
  a.weighted = 0;
  a.add = 0;
  a.ptr_off = 0;
  a.nmaps_run = P->nmaps;
  a.pair0 = 0;
  a.npairs_run = P->npairs;
  a.m_identity = P->m_identity;
  return a;
}

cudaError_t launch_fft_syn(const sht_plan_s *P, const DevPtrs &map, int polar, int weighted, int add,
                           cudaStream_t st, int p0, int p1) {
  if (p1 < 0) p1 = P->npairs;
  if (p1 <= p0) return cudaSuccess;
  FftArgs a = make_fft_args(P, map, polar);
  a.weighted = weighted;
  a.add = add;
  a.pair0 = p0;
  a.npairs_run = p1 - p0;
  const bool df = P->fft_df;
  if (P->d_fft_scratch) {
    const int g = (int)std::min<int64_t>((int64_t)a.npairs_run * P->nmaps, P->fft_slots);
    if (df)
      fft_syn_kernel_global<DF><<<g, kFftThreads, 0, st>>>(a, P->d_fft_scratch, P->fft_slot_len);
    else
      fft_syn_kernel_global<F64><<<g, kFftThreads, 0, st>>>(a, P->d_fft_scratch, P->fft_slot_len);
    return cudaGetLastError();
  }
  dim3 grid(a.npairs_run, P->nmaps);
  if (df)
    fft_syn_kernel<DF><<<grid, kFftThreads, P->fft_smem, st>>>(a);
  else
    fft_syn_kernel<F64><<<grid, kFftThreads, P->fft_smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fft_ana(const sht_plan_s *P, const DevPtrs &map, int weighted, cudaStream_t st, int p0,
                           int p1) {
  if (p1 < 0) p1 = P->npairs;
  if (p1 <= p0) return cudaSuccess;
  FftArgs a = make_fft_args(P, map, 1);
  a.weighted = weighted;
  a.pair0 = p0;
  a.npairs_run = p1 - p0;
  const bool df = P->fft_df;
  if (P->d_fft_scratch) {
    const int g = (int)std::min<int64_t>((int64_t)a.npairs_run * P->nmaps, P->fft_slots);
    if (df)
      fft_ana_kernel_global<DF><<<g, kFftThreads, 0, st>>>(a, P->d_fft_scratch, P->fft_slot_len);
    else
      fft_ana_kernel_global<F64><<<g, kFftThreads, 0, st>>>(a, P->d_fft_scratch, P->fft_slot_len);
    return cudaGetLastError();
  }
  dim3 grid(a.npairs_run, P->nmaps);
  if (df)
    fft_ana_kernel<DF><<<grid, kFftThreads, P->fft_smem, st>>>(a);
  else
    fft_ana_kernel<F64><<<grid, kFftThreads, P->fft_smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sht

// ---------------------------------------------------------------------------
// batches (sht_batch_execute)
// ---------------------------------------------------------------------------
namespace sht {

size_t fft_args_size() { return sizeof(FftArgs); }

void fft_fill_args(const sht_plan_s *P, int polar, int weighted, int add, int ptr_off, void *out) {
  DevPtrs none;
  memset(&none, 0, sizeof(none));
  FftArgs a = make_fft_args(P, none, polar);
  a.weighted = weighted;
  a.add = add;
  a.ptr_off = ptr_off;
  memcpy(out, &a, sizeof(a));
}

cudaError_t fft_prepare_device(int device) {
  static std::mutex mu;
  static std::set<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(device)) return cudaSuccess;
  int smem = 0;
  cudaError_t e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess) {  // radix constants, from long double
    static double hc[kMaxRadix + 1][kMaxRadix / 2 + 1], hs[kMaxRadix + 1][kMaxRadix / 2 + 1];
    static float2 hc2[kMaxRadix + 1][kMaxRadix / 2 + 1], hs2[kMaxRadix + 1][kMaxRadix / 2 + 1];
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int R = 3; R <= kMaxRadix; R += 2)
      for (int t = 1; t <= R / 2; ++t) {
        const long double c = cosl(2.0L * pi * t / R), s = sinl(2.0L * pi * t / R);
        hc[R][t] = (double)c;
        hs[R][t] = (double)s;
        hc2[R][t] = make_float2((float)c, (float)(c - (float)c));
        hs2[R][t] = make_float2((float)s, (float)(s - (float)s));
      }
    e = cudaMemcpyToSymbol(c_cos, hc, sizeof(hc));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sin, hs, sizeof(hs));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cos2, hc2, sizeof(hc2));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sin2, hs2, sizeof(hs2));
  }
  const void *fns[9] = {(const void *)fft_syn_kernel<F64>,       (const void *)fft_ana_kernel<F64>,
                        (const void *)fft_syn_kernel_batch<F64>, (const void *)fft_ana_kernel_batch<F64>,
                        (const void *)fft_syn_kernel<DF>,        (const void *)fft_ana_kernel<DF>,
                        (const void *)fft_syn_kernel_batch<DF>,  (const void *)fft_ana_kernel_batch<DF>,
                        (const void *)spectrum_kernel};
  for (int i = 0; i < 9 && e == cudaSuccess; ++i) {
    // static + dynamic shared memory may not exceed the opt-in size
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fns[i]);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, smem - (int)fa.sharedSizeBytes);
  }
  if (e == cudaSuccess) done.insert(device);
  return e;
}

// synthesis (stage 0) or analysis (stage 1) ring FFTs of every item (pair, map, -, args index),
// in double-float (df: items of mixed plans) or FP64
cudaError_t launch_fft_batch(int stage, bool df, const void *args, const int4 *items, int n, int smem,
                             const PtrTable &tbl, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const FftArgs *a = static_cast<const FftArgs *>(args);
  if (stage == 0) {
    if (df)
      fft_syn_kernel_batch<DF><<<n, kFftThreads, smem, st>>>(a, items, tbl);
    else
      fft_syn_kernel_batch<F64><<<n, kFftThreads, smem, st>>>(a, items, tbl);
  } else {
    if (df)
      fft_ana_kernel_batch<DF><<<n, kFftThreads, smem, st>>>(a, items, tbl);
    else
      fft_ana_kernel_batch<F64><<<n, kFftThreads, smem, st>>>(a, items, tbl);
  }
  return cudaGetLastError();
}

}  // namespace sht
