// fft.cu -- ring FFTs of Eqs. syn1 and ana2 in IEEE double.
//
// One CTA transforms one north/south ring pair of one map: the two real
// rings are packed as z = p_north + i p_south into a single complex DFT of
// length Nphi (pairs always share Nphi).  The whole ring lives in shared
// memory; the engine is a mixed-radix Stockham (autosort) transform whose
// passes compute every output of a radix-R butterfly directly (R multiply-
// adds per output, twiddles from a table), so any radix works the same way.
// Lengths with a prime factor above 31 go through Rader's algorithm (prime
// n, n-1 smooth: a cyclic convolution of length n-1) or Bluestein's (chirp
// convolution of power-of-two length >= 2n-1).
//
// Synthesis, per ring:  p_x = sum_{m=-mmax}^{mmax} c_m e^{2 pi i m x / N},
//   c_m = F_m e^{i m phi0} (m >= 0), c_{-m} = conj(c_m); m is folded modulo N
//   when N <= 2 mmax (aliasing, Eq. syn1).
// Analysis, per ring:   G_m = w e^{-i m phi0} sum_x p_x e^{-2 pi i m x / N}  (Eq. ana2).
#include <mutex>
#include <set>

#include "sht_internal.h"

namespace sht {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// One Stockham pass of radix R over buf[0..len) (forward, e^{-i}).
// Output o = (j / Ns) Ns R + s Ns + (j % Ns) receives
//   sum_r buf[j + r len/R] W^{r (k len/(Ns R) + s len/R)},  k = j % Ns.
__device__ void fft_pass(double2 *buf, int len, int R, int Ns, const double2 *__restrict__ W) {
  double2 out[kFftMaxOpt];
  const int nt = blockDim.x;
  const int step = len / R;
  const int NsR = Ns * R;
  const int tws = len / NsR;
#pragma unroll
  for (int i = 0; i < kFftMaxOpt; ++i) {
    const int o = threadIdx.x + i * nt;
    if (o < len) {
      const int q = o / NsR;
      const int rem = o - q * NsR;
      const int s = rem / Ns;
      const int k = rem - s * Ns;
      const int j = q * Ns + k;
      const int base = k * tws + s * step;  // < len
      double2 acc = buf[j];
      int t = 0;
      for (int r = 1; r < R; ++r) {
        t += base;
        if (t >= len) t -= len;
        acc = cadd(acc, cmul(buf[j + r * step], __ldg(W + t)));
      }
      out[i] = acc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kFftMaxOpt; ++i) {
    const int o = threadIdx.x + i * nt;
    if (o < len) buf[o] = out[i];
  }
  __syncthreads();
}

__device__ void fft_forward(double2 *buf, const FftPlanDev &fp) {
  int Ns = 1;
  for (int i = 0; i < fp.nrad; ++i) {
    fft_pass(buf, fp.len, fp.rad[i], Ns, fp.w);
    Ns *= fp.rad[i];
  }
}

// Full forward DFT of length n of the data placed by the caller:
//   kind 0: buf[k] = x_k (k < n);
//   kind 1: buf[q] = x_{g^q} (q < n-1), *x0 = x_0;
//   kind 2: buf[k] = x_k chirp_k (k < n), 0 up to len.
// Afterwards dft_at(k) returns X_k.
__device__ void dft_run(double2 *buf, const FftPlanDev &fp, double2 *sh_x0, double2 *sh_a0) {
  fft_forward(buf, fp);
  if (fp.kind == 0) return;
  if (fp.kind == 1 && threadIdx.x == 0) *sh_a0 = buf[0];
  __syncthreads();
  // multiply by the kernel spectrum and transform back: IDFT(y) = conj(DFT(conj(y)))
  for (int i = threadIdx.x; i < fp.len; i += blockDim.x) buf[i] = cconj(cmul(buf[i], fp.spec[i]));
  __syncthreads();
  fft_forward(buf, fp);
}

__device__ __forceinline__ double2 dft_at(const double2 *buf, const FftPlanDev &fp, int k, double2 x0,
                                          double2 a0) {
  if (fp.kind == 0) return buf[k];
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
  extern __shared__ double2 buf[];
  const FftPlanDev fp = *fpd;
  for (int i = threadIdx.x; i < len; i += blockDim.x) buf[i] = src[i];
  __syncthreads();
  fft_forward(buf, fp);
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = make_double2(buf[i].x * scale, buf[i].y * scale);
}

cudaError_t launch_fft_spectrum(const FftPlanDev *hp, const FftPlanDev *dp, const double2 *src, double2 *dst,
                                int len, double scale, cudaStream_t st) {
  const int smem = len * (int)sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(spectrum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  spectrum_kernel<<<1, kFftThreads, smem, st>>>(dp, src, dst, len, scale);
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

__device__ __forceinline__ void fft_syn_kernel_body(const FftArgs &a, double *const *ptrs, const int p, const int j) {
  extern __shared__ double2 buf[];
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
  dft_run(buf, fp, &sh_x0, &sh_a0);
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
__global__ void __launch_bounds__(kFftThreads) fft_syn_kernel(FftArgs a) {
  fft_syn_kernel_body(a, a.map.p, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(kFftThreads) fft_syn_kernel_batch(const FftArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const FftArgs &a = args[it.w];
  fft_syn_kernel_body(a, tbl.p + a.ptr_off, it.x, it.y);
}

// ---------------------------------------------------------------------------
// analysis: ring pixels -> G (per m)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fft_ana_kernel_body(const FftArgs &a, double *const *ptrs, const int p, const int j) {
  extern __shared__ double2 buf[];
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
  dft_run(buf, fp, &sh_x0, &sh_a0);
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
__global__ void __launch_bounds__(kFftThreads) fft_ana_kernel(FftArgs a) {
  fft_ana_kernel_body(a, a.map.p, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(kFftThreads) fft_ana_kernel_batch(const FftArgs *__restrict__ args,
    const int4 *__restrict__ items, const PtrTable tbl) {
  const int4 it = items[blockIdx.x];
  const FftArgs &a = args[it.w];
  fft_ana_kernel_body(a, tbl.p + a.ptr_off, it.x, it.y);
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
  return a;
}

cudaError_t launch_fft_syn(const sht_plan_s *P, const DevPtrs &map, int polar, int weighted, int add,
                           cudaStream_t st) {
  FftArgs a = make_fft_args(P, map, polar);
  a.weighted = weighted;
  a.add = add;
  dim3 grid(P->npairs, P->nmaps);
  fft_syn_kernel<<<grid, kFftThreads, P->fft_smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fft_ana(const sht_plan_s *P, const DevPtrs &map, int weighted, cudaStream_t st) {
  FftArgs a = make_fft_args(P, map, 1);
  a.weighted = weighted;
  dim3 grid(P->npairs, P->nmaps);
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
  const void *fns[4] = {(const void *)fft_syn_kernel, (const void *)fft_ana_kernel,
                        (const void *)fft_syn_kernel_batch, (const void *)fft_ana_kernel_batch};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
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
