// fft.cu -- ring FFTs of Eqs. syn1 and ana2 in IEEE double.
//
// One CTA transforms one north/south ring pair of one map: the two real
// rings are packed as z = p_north + i p_south into a single complex DFT of
// length Nphi (pairs always share Nphi).  The ring lives in shared memory
// (up to kFftMaxLen points; longer rings in an L2-resident global scratch slot
// per CTA of a persistent grid) and is transformed in place: mixed-radix
// decimation-in-frequency
// passes (radix 2, 4 and odd radices up to 31 with each thread running whole
// butterflies, one barrier per pass; odd radices up to 127 as sweeps over the
// ring); the output comes out digit-reversed and
// is read back through a position table.  Lengths with a prime factor above
// 127 go through Rader's algorithm (prime n, n-1 smooth: a cyclic convolution
// of length n-1) or Bluestein's (chirp convolution of smooth length >= 2n-1);
// both convolutions run DIF forward and the transposed (DIT) passes back, so
// the result returns to natural order without a permutation pass.
//
// Synthesis, per ring:  p_x = sum_{m=-mmax}^{mmax} c_m e^{2 pi i m x / N},
//   c_m = F_m e^{i m phi0} (m >= 0), c_{-m} = conj(c_m); m is folded modulo N
//   when N <= 2 mmax (aliasing, Eq. syn1).
// Analysis, per ring:   G_m = w e^{-i m phi0} sum_x p_x e^{-2 pi i m x / N}  (Eq. ana2).
#include <algorithm>
#include <mutex>
#include <set>

#include "sht_internal.h"

namespace sht {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// cos(2 pi t / R) and sin(2 pi t / R) for odd radices R <= kMaxRadix, t = 1..(R-1)/2,
// written once per device (fft_prepare_device).  The butterflies index them with
// compile-time constants, so they are read as constant-bank operands.
__constant__ double c_cos[kMaxRadix + 1][kMaxRadix / 2 + 1];
__constant__ double c_sin[kMaxRadix + 1][kMaxRadix / 2 + 1];

// y_s = sum_r x_r e^{-2 pi i r s / R} for s < R; out(s, y_s) receives each output.
// Odd R uses the symmetric form: with S_j = x_j + x_{R-j}, D_j = x_j - x_{R-j},
//   y_k = A_k - i B_k,  y_{R-k} = A_k + i B_k,
//   A_k = x_0 + sum_j S_j cos(2 pi j k / R),  B_k = sum_j D_j sin(2 pi j k / R),
// i.e. 4 h^2 real multiply-adds for R points (h = (R-1)/2) instead of 4 R^2.
template <int R, class Out>
__device__ __forceinline__ void dft_small(double2 (&x)[R], Out &&out) {
  if constexpr (R == 2) {
    out(0, cadd(x[0], x[1]));
    out(1, csub(x[0], x[1]));
  } else if constexpr (R == 4) {
    const double2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
    const double2 s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
    out(0, cadd(s02, s13));
    out(1, make_double2(d02.x + d13.y, d02.y - d13.x));  // d02 - i d13
    out(2, csub(s02, s13));
    out(3, make_double2(d02.x - d13.y, d02.y + d13.x));  // d02 + i d13
  } else {
    static_assert(R % 2 == 1 && R <= kMaxRadix, "odd radix");
    constexpr int h = (R - 1) / 2;
    const double2 x0 = x[0];
    double2 y0 = x0;
#pragma unroll
    for (int j = 1; j <= h; ++j) {  // S_j into x[j], D_j into x[R-j]
      const double2 a = x[j], b = x[R - j];
      x[j] = cadd(a, b);
      x[R - j] = csub(a, b);
      y0 = cadd(y0, x[j]);
    }
    out(0, y0);
#pragma unroll
    for (int k = 1; k <= h; ++k) {
      double2 A = x0, B = make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 1; j <= h; ++j) {
        const int t = (j * k) % R;
        const double c = t <= h ? c_cos[R][t] : c_cos[R][R - t];
        const double sn = t <= h ? c_sin[R][t] : -c_sin[R][R - t];
        A.x = fma(x[j].x, c, A.x);
        A.y = fma(x[j].y, c, A.y);
        B.x = fma(x[R - j].x, sn, B.x);
        B.y = fma(x[R - j].y, sn, B.y);
      }
      out(k, make_double2(A.x + B.y, A.y - B.x));
      out(R - k, make_double2(A.x - B.y, A.y + B.x));
    }
  }
}

// The ring buffer: the kernels' dynamic shared memory, named at namespace scope
// so the out-of-line passes address it as shared memory.
extern __shared__ double2 s_ring[];

// Where a ring lives while it is transformed: shared memory (every length up to
// kFftMaxLen), or a CTA-private slot of global scratch for longer rings, which
// stays in L2 (the engine is the same; barriers order global accesses within
// the CTA as they do shared ones).
struct SharedRing {
  __device__ __forceinline__ double2 *at(int i) const { return s_ring + i; }
};
struct GlobalRing {
  double2 *p;
  __device__ __forceinline__ double2 *at(int i) const { return p + i; }
};

// One in-place pass of radix R over the len / L blocks of length L of the ring.
// Butterfly (block B, offset b < L/R) works on ring[B L + b + r L/R], r < R:
//   decimation in frequency (DIT = false): DFT_R, then output s times W_L^{s b};
//   its transpose (DIT = true): input r times W_L^{r b}, then DFT_R.
// Each butterfly touches only its own R slots, so one barrier per pass suffices.
// W holds e^{-2 pi i k / len}; W_L^e = W[e len / L].
template <int R, bool DIT, class Ring>
__device__ __noinline__ void fft_stage(Ring ring, int len, int L, const double2 *__restrict__ W) {
  const int LR = L / R;
  const int nb = len / R;
  const int tw = len / L;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) {
    const int B = q / LR, b = q - B * LR;
    double2 *p = ring.at(B * L + b);
    double2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = p[r * LR];
    if (DIT && b != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], __ldg(W + r * b * tw));
    }
    dft_small<R>(x, [&](int s, double2 y) {
      if (!DIT && s != 0 && b != 0) y = cmul(y, __ldg(W + s * b * tw));
      p[s * LR] = y;
    });
  }
  __syncthreads();
}

// One in-place pass of an odd radix R in (kMaxRadix, kMaxBigRadix], the same
// butterflies as fft_stage.  R values no longer fit in one thread's registers, so
// the symmetric form of dft_small runs as sweeps over the ring:
//   1. S_j = x_j + x_{R-j} into slot j and D_j = x_j - x_{R-j} into slot R-j
//      (j = 1..h, after the input twiddles for DIT), one item per (butterfly, j);
//   2. in rounds of whole butterflies, one item per (butterfly, k), k = 0..h,
//      computes y_k and y_{R-k} from x_0, S and D into registers; after a barrier
//      the items write them back in place (DIF: times the output twiddles).
// Items are k-major so that a warp shares k (its cos/sin loads broadcast) and
// walks consecutive butterflies (consecutive slots).  cos and sin of 2 pi t / R
// come from the ring's own table: W[t len / R] = e^{-2 pi i t / R}.
template <bool DIT, class Ring>
__device__ __noinline__ void fft_stage_big(Ring ring, int len, int L, int R, const double2 *__restrict__ W) {
  constexpr int kItems = 4;  // output pairs a thread holds across the barrier
  const int LR = L / R, nb = len / R, tw = len / L, h = (R - 1) / 2, tr = len / R;
  for (int i = threadIdx.x; i < nb * h; i += blockDim.x) {
    const int j = 1 + i / nb, q = i % nb;
    const int B = q / LR, b = q - B * LR;
    double2 *p = ring.at(B * L + b);
    double2 u = p[j * LR], v = p[(R - j) * LR];
    if (DIT && b != 0) {
      u = cmul(u, __ldg(W + j * b * tw));
      v = cmul(v, __ldg(W + (R - j) * b * tw));
    }
    p[j * LR] = cadd(u, v);
    p[(R - j) * LR] = csub(u, v);
  }
  __syncthreads();
  const int per = h + 1;
  int nround = (int)(blockDim.x * kItems) / per;  // butterflies per round
  if (nround >= 32) nround &= ~31;
  for (int q0 = 0; q0 < nb; q0 += nround) {
    const int nq = min(nround, nb - q0), nit = nq * per;
    double2 ya[kItems], yb[kItems];
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
      const int i = threadIdx.x + u * blockDim.x;
      if (i < nit) {
        const int k = i / nq, q = q0 + i % nq;
        const int B = q / LR, b = q - B * LR;
        const double2 *p = ring.at(B * L + b);
        double2 A = p[0];
        if (k == 0) {
          for (int j = 1; j <= h; ++j) A = cadd(A, p[j * LR]);
          ya[u] = A;
        } else {
          double2 Bn = make_double2(0.0, 0.0);  // -(sum_j D_j sin(2 pi j k / R))
          int t = 0;
          for (int j = 1; j <= h; ++j) {
            t += k;
            if (t >= R) t -= R;
            const double2 w = __ldg(W + t * tr);
            const double2 sj = p[j * LR], dj = p[(R - j) * LR];
            A.x = fma(sj.x, w.x, A.x);
            A.y = fma(sj.y, w.x, A.y);
            Bn.x = fma(dj.x, w.y, Bn.x);
            Bn.y = fma(dj.y, w.y, Bn.y);
          }
          ya[u] = make_double2(A.x - Bn.y, A.y + Bn.x);  // y_k = A - i B
          yb[u] = make_double2(A.x + Bn.y, A.y - Bn.x);  // y_{R-k} = A + i B
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
        double2 *p = ring.at(B * L + b);
        double2 y0 = ya[u];
        if (k == 0) {
          p[0] = y0;
        } else {
          double2 y1 = yb[u];
          if (!DIT && b != 0) {
            y0 = cmul(y0, __ldg(W + k * b * tw));
            y1 = cmul(y1, __ldg(W + (R - k) * b * tw));
          }
          p[k * LR] = y0;
          p[(R - k) * LR] = y1;
        }
      }
    }
    __syncthreads();
  }
}

template <bool DIT, class Ring>
__device__ void fft_stage_any(Ring ring, int len, int L, int R, const double2 *W) {
  switch (R) {
    case 2: fft_stage<2, DIT>(ring, len, L, W); break;
    case 3: fft_stage<3, DIT>(ring, len, L, W); break;
    case 4: fft_stage<4, DIT>(ring, len, L, W); break;
    case 5: fft_stage<5, DIT>(ring, len, L, W); break;
    case 7: fft_stage<7, DIT>(ring, len, L, W); break;
    case 11: fft_stage<11, DIT>(ring, len, L, W); break;
    case 13: fft_stage<13, DIT>(ring, len, L, W); break;
    case 17: fft_stage<17, DIT>(ring, len, L, W); break;
    case 19: fft_stage<19, DIT>(ring, len, L, W); break;
    case 23: fft_stage<23, DIT>(ring, len, L, W); break;
    case 29: fft_stage<29, DIT>(ring, len, L, W); break;
    case 31: fft_stage<31, DIT>(ring, len, L, W); break;
    default: fft_stage_big<DIT>(ring, len, L, R, W); break;
  }
}

// Forward DFT of ring[0..fp.len) by decimation in frequency: natural-order input,
// output X_k at position fp.pos[k] (mixed-radix digit reversal).
template <class Ring>
__device__ void fft_dif(Ring ring, const FftPlanDev &fp) {
  int L = fp.len;
  for (int i = 0; i < fp.nrad; ++i) {
    fft_stage_any<false>(ring, fp.len, L, fp.rad[i], fp.w);
    L /= fp.rad[i];
  }
}

// The transpose of fft_dif (its passes transposed, in reverse order): input
// z_k at position fp.pos[k], output the forward DFT of z in natural order.
template <class Ring>
__device__ void fft_dit(Ring ring, const FftPlanDev &fp) {
  int L = 1;
  for (int i = fp.nrad - 1; i >= 0; --i) {
    L *= fp.rad[i];
    fft_stage_any<true>(ring, fp.len, L, fp.rad[i], fp.w);
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
template <class Ring>
__device__ void dft_run(Ring ring, const FftPlanDev &fp, double2 *sh_x0, double2 *sh_a0) {
  double2 *const buf = ring.at(0);
  fft_dif(ring, fp);
  if (fp.kind == 0) return;
  if (fp.kind == 1 && threadIdx.x == 0) *sh_a0 = buf[0];  // X_0 sits at position 0
  __syncthreads();
  for (int i = threadIdx.x; i < fp.len; i += blockDim.x) buf[i] = cconj(cmul(buf[i], fp.spec[i]));
  __syncthreads();
  fft_dit(ring, fp);
}

__device__ __forceinline__ double2 dft_at(const double2 *buf, const FftPlanDev &fp, int k, double2 x0,
                                          double2 a0) {
  if (fp.kind == 0) return buf[__ldg(fp.pos + k)];
  if (fp.kind == 1) {
    if (k == 0) return cadd(x0, a0);
    return cadd(x0, cconj(buf[fp.inv_out[k]]));
  }
  return cmul(fp.chirp[k], cconj(buf[k]));
}

// ---------------------------------------------------------------------------
// spectrum precomputation (plan time): dst = scale * DFT_len(src)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFftThreads) spectrum_kernel(const FftPlanDev *fpd, const double2 *src,
                                                              double2 *dst, int len, double scale) {
  double2 *const buf = s_ring;
  const FftPlanDev fp = *fpd;
  for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = src[i];
  __syncthreads();
  fft_dif(SharedRing{}, fp);
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = make_double2(buf[i].x * scale, buf[i].y * scale);
}
// the same for lengths beyond shared memory: transformed in place in dst
__global__ void __launch_bounds__(kFftThreads) spectrum_kernel_global(const FftPlanDev *fpd, const double2 *src,
                                                                     double2 *dst, int len, double scale) {
  const FftPlanDev fp = *fpd;
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  fft_dif(GlobalRing{dst}, fp);
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

// e^{i m phi0} with the product m*phi0 carried to ~1e-32 before the sincos
__device__ __forceinline__ double2 phase_of(int m, double phi0) {
  if (phi0 == 0.0 || m == 0) return make_double2(1.0, 0.0);
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
};

// ---------------------------------------------------------------------------
// synthesis: F (per m) -> ring pixels
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 synth_coef(const FftArgs &a, int j, int p, int m, double phi_n, double phi_s,
                                              bool south, bool conj_) {
  // cN + i cS for coefficient m of the two rings (conj_: conj(cN) + i conj(cS));
  // F below the first pair the Legendre stage processed for this m is zero.
  const int mi = a.minv[m];
  if (mi < 0 || p < a.syn_first[mi]) return make_double2(0.0, 0.0);
  const double2 *f = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
  double2 cn = cmul(f[0], phase_of(m, phi_n));
  double2 cs = south ? cmul(f[1], phase_of(m, phi_s)) : make_double2(0.0, 0.0);
  if (conj_) {
    cn = cconj(cn);
    cs = cconj(cs);
  }
  return make_double2(cn.x - cs.y, cn.y + cs.x);
}

// Z_k = sum_{m >= 0, m = k mod N} (cN_m + i cS_m) + sum_{m >= 1, -m = k mod N} (conj cN_m + i conj cS_m)
__device__ double2 spectrum_at(const FftArgs &a, int j, int p, int k, int N, double phi_n, double phi_s,
                               bool south) {
  double2 z = make_double2(0.0, 0.0);
  for (int m = k; m <= a.mmax; m += N) z = cadd(z, synth_coef(a, j, p, m, phi_n, phi_s, south, false));
  for (int m = (k == 0 ? N : N - k); m <= a.mmax; m += N)
    z = cadd(z, synth_coef(a, j, p, m, phi_n, phi_s, south, true));
  return z;
}

template <class Ring>
__device__ __forceinline__ void fft_syn_kernel_body(Ring ring, const FftArgs &a, double *const *ptrs, const int p,
                                     const int j) {
  double2 *const buf = ring.at(0);
  __shared__ double2 sh_x0, sh_a0;
  const FftPlanDev fp = a.plans[a.pair_fft[p]];
  const int2 rr = a.pair_rings[p];
  const RingDev rn = a.rings[rr.x];
  const bool south = rr.y >= 0;
  const RingDev rs = a.rings[south ? rr.y : rr.x];
  const int N = fp.n;
  // inverse DFT via conj(DFT(conj(Z)))
  if (fp.kind == 0) {
    for (int k = threadIdx.x; k < N; k += blockDim.x)
      buf[k] = cconj(spectrum_at(a, j, p, k, N, rn.phi0, rs.phi0, south));
  } else if (fp.kind == 1) {
    for (int q = threadIdx.x; q < N - 1; q += blockDim.x)
      buf[q] = cconj(spectrum_at(a, j, p, fp.perm_in[q], N, rn.phi0, rs.phi0, south));
    if (threadIdx.x == 0) sh_x0 = cconj(spectrum_at(a, j, p, 0, N, rn.phi0, rs.phi0, south));
  } else {
    for (int k = threadIdx.x; k < fp.len; k += blockDim.x)
      buf[k] = (k < N) ? cmul(cconj(spectrum_at(a, j, p, k, N, rn.phi0, rs.phi0, south)), fp.chirp[k])
                       : make_double2(0.0, 0.0);
  }
  __syncthreads();
  dft_run(ring, fp, &sh_x0, &sh_a0);
  const double2 x0 = sh_x0, a0 = sh_a0;
  double *mp = ptrs[j];
  const double wn = a.weighted ? rn.weight : 1.0, ws = a.weighted ? rs.weight : 1.0;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const double2 X = dft_at(buf, fp, x, x0, a0);
    // z = conj(X): north = Re z, south = Im z
    double vn = X.x * wn;
    double *on = mp + rn.ofs + (int64_t)x * rn.stride;
    if (a.add) vn += *on;
    *on = vn;
    if (south) {
      double vs = -X.y * ws;
      double *os = mp + rs.ofs + (int64_t)x * rs.stride;
      if (a.add) vs += *os;
      *os = vs;
    }
  }
}
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_syn_kernel(FftArgs a) {
  fft_syn_kernel_body(SharedRing{}, a, a.map.p, a.pair0 + blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_syn_kernel_batch(const FftArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const FftArgs &a = args[it.w];
  fft_syn_kernel_body(SharedRing{}, a, tbl.p + a.ptr_off, it.x, it.y);
}

// ---------------------------------------------------------------------------
// analysis: ring pixels -> G (per m)
// ---------------------------------------------------------------------------
template <class Ring>
__device__ __forceinline__ void fft_ana_kernel_body(Ring ring, const FftArgs &a, double *const *ptrs, const int p,
                                     const int j) {
  double2 *const buf = ring.at(0);
  __shared__ double2 sh_x0, sh_a0;
  const FftPlanDev fp = a.plans[a.pair_fft[p]];
  const int2 rr = a.pair_rings[p];
  const RingDev rn = a.rings[rr.x];
  const bool south = rr.y >= 0;
  const RingDev rs = a.rings[south ? rr.y : rr.x];
  const int N = fp.n;
  const double *mp = ptrs[j];
  auto zin = [&](int x) {
    const double vn = mp[rn.ofs + (int64_t)x * rn.stride];
    const double vs = south ? mp[rs.ofs + (int64_t)x * rs.stride] : 0.0;
    return make_double2(vn, vs);
  };
  if (fp.kind == 0) {
    for (int k = threadIdx.x; k < N; k += blockDim.x) buf[k] = zin(k);
  } else if (fp.kind == 1) {
    for (int q = threadIdx.x; q < N - 1; q += blockDim.x) buf[q] = zin(fp.perm_in[q]);
    if (threadIdx.x == 0) sh_x0 = zin(0);
  } else {
    for (int k = threadIdx.x; k < fp.len; k += blockDim.x)
      buf[k] = (k < N) ? cmul(zin(k), fp.chirp[k]) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  dft_run(ring, fp, &sh_x0, &sh_a0);
  const double2 x0 = sh_x0, a0 = sh_a0;
  const double wn = a.weighted ? rn.weight : 1.0, ws = a.weighted ? rs.weight : 1.0;
  for (int mi = threadIdx.x; mi < a.nm; mi += blockDim.x) {
    const int m = a.mval[mi];
    const int k = m % N, kn = (N - k) % N;
    const double2 Zk = dft_at(buf, fp, k, x0, a0), Zn = cconj(dft_at(buf, fp, kn, x0, a0));
    // P_N = (Zk + conj Zn)/2,  P_S = (Zk - conj Zn)/(2i)
    const double2 pn = make_double2(0.5 * (Zk.x + Zn.x), 0.5 * (Zk.y + Zn.y));
    const double2 d = make_double2(Zk.x - Zn.x, Zk.y - Zn.y);
    const double2 ps = make_double2(0.5 * d.y, -0.5 * d.x);
    const double2 en = cconj(phase_of(m, rn.phi0)), es = cconj(phase_of(m, rs.phi0));
    double2 gn = cmul(pn, en), gs = cmul(ps, es);
    gn.x *= wn;
    gn.y *= wn;
    gs.x *= ws;
    gs.y *= ws;
    if (!south) gs = make_double2(0.0, 0.0);
    double2 *g = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
    g[0] = gn;
    g[1] = gs;
  }
}
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_ana_kernel(FftArgs a) {
  fft_ana_kernel_body(SharedRing{}, a, a.map.p, a.pair0 + blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(kFftThreads, kFftMinBlocks) fft_ana_kernel_batch(const FftArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const FftArgs &a = args[it.w];
  fft_ana_kernel_body(SharedRing{}, a, tbl.p + a.ptr_off, it.x, it.y);
}

// Rings longer than shared memory holds: a persistent grid, each CTA owning one
// scratch slot of slot_len points, walks the (pair, map) items in turn.
__global__ void __launch_bounds__(kFftThreads) fft_syn_kernel_global(FftArgs a, double2 *scratch,
                                                                     int slot_len) {
  const GlobalRing ring{scratch + (size_t)blockIdx.x * slot_len};
  const int n = a.npairs_run * a.nmaps_run;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    fft_syn_kernel_body(ring, a, a.map.p, a.pair0 + it % a.npairs_run, it / a.npairs_run);
    __syncthreads();  // the slot is rewritten by the next item
  }
}
__global__ void __launch_bounds__(kFftThreads) fft_ana_kernel_global(FftArgs a, double2 *scratch,
                                                                     int slot_len) {
  const GlobalRing ring{scratch + (size_t)blockIdx.x * slot_len};
  const int n = a.npairs_run * a.nmaps_run;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    fft_ana_kernel_body(ring, a, a.map.p, a.pair0 + it % a.npairs_run, it / a.npairs_run);
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
  if (P->d_fft_scratch) {
    const int g = (int)std::min<int64_t>((int64_t)a.npairs_run * P->nmaps, P->fft_slots);
    fft_syn_kernel_global<<<g, kFftThreads, 0, st>>>(a, P->d_fft_scratch, P->fft_slot_len);
    return cudaGetLastError();
  }
  dim3 grid(a.npairs_run, P->nmaps);
  fft_syn_kernel<<<grid, kFftThreads, P->fft_smem, st>>>(a);
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
  if (P->d_fft_scratch) {
    const int g = (int)std::min<int64_t>((int64_t)a.npairs_run * P->nmaps, P->fft_slots);
    fft_ana_kernel_global<<<g, kFftThreads, 0, st>>>(a, P->d_fft_scratch, P->fft_slot_len);
    return cudaGetLastError();
  }
  dim3 grid(a.npairs_run, P->nmaps);
  fft_ana_kernel<<<grid, kFftThreads, P->fft_smem, st>>>(a);
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
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int R = 3; R <= kMaxRadix; R += 2)
      for (int t = 1; t <= R / 2; ++t) {
        hc[R][t] = (double)cosl(2.0L * pi * t / R);
        hs[R][t] = (double)sinl(2.0L * pi * t / R);
      }
    e = cudaMemcpyToSymbol(c_cos, hc, sizeof(hc));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sin, hs, sizeof(hs));
  }
  const void *fns[5] = {(const void *)fft_syn_kernel, (const void *)fft_ana_kernel,
                        (const void *)fft_syn_kernel_batch, (const void *)fft_ana_kernel_batch,
                        (const void *)spectrum_kernel};
  for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
    // static + dynamic shared memory may not exceed the opt-in size
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fns[i]);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, smem - (int)fa.sharedSizeBytes);
  }
  if (e == cudaSuccess) done.insert(device);
  return e;
}

// synthesis (stage 0) or analysis (stage 1) ring FFTs of every item (pair, map, -, args index)
cudaError_t launch_fft_batch(int stage, const void *args, const int4 *items, int n, int smem, const PtrTable &tbl,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const FftArgs *a = static_cast<const FftArgs *>(args);
  if (stage == 0)
    fft_syn_kernel_batch<<<n, kFftThreads, smem, st>>>(a, items, tbl);
  else
    fft_ana_kernel_batch<<<n, kFftThreads, smem, st>>>(a, items, tbl);
  return cudaGetLastError();
}

}  // namespace sht
