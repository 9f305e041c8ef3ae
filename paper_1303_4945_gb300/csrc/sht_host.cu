// sht_host.cu -- C ABI entry points: geometry, a_lm layout, plans, execution.
//
// Host code only plans (ring pairing, polar-cut ranges, work lists, FFT
// factorisations) and launches; every step of a transform runs in the CUDA
// kernels of legendre_*.cu and fft.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <map>
#include <numeric>

#include "sht_internal.h"

using namespace sht;

// ----------------------------------------------------------------------------
// Errors
// ----------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int sht::set_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      if (e_ == cudaErrorMemoryAllocation) return fail(SHT_ERR_OOM, "%s: %s", #expr, cudaGetErrorString(e_)); \
      return fail(SHT_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));               \
    }                                                                                   \
  } while (0)

extern "C" const char *sht_strerror(int code) {
  switch (code) {
    case SHT_OK: return "ok";
    case SHT_ERR_INVALID_ARG: return "invalid argument";
    case SHT_ERR_UNSUPPORTED: return "unsupported";
    case SHT_ERR_OOM: return "out of memory";
    case SHT_ERR_CUDA: return "CUDA error";
    case SHT_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

extern "C" const char *sht_last_error(void) { return g_last_error.c_str(); }

// ----------------------------------------------------------------------------
// Geometry
// ----------------------------------------------------------------------------
static const long double kPiL = 3.141592653589793238462643383279502884L;

extern "C" int sht_geom_general(int nrings, const double *theta, const int *nphi, const double *phi0,
                                const int64_t *ofs, const int *stride, const double *weight,
                                sht_geom_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nrings < 1 || !theta || !nphi || !phi0 || !ofs)
    return fail(SHT_ERR_INVALID_ARG, "nrings < 1 or a required array is NULL");
  for (int i = 0; i < nrings; ++i) {
    if (!(theta[i] >= 0.0 && theta[i] <= M_PI)) return fail(SHT_ERR_INVALID_ARG, "theta[%d] outside [0, pi]", i);
    if (nphi[i] < 1) return fail(SHT_ERR_INVALID_ARG, "nphi[%d] < 1", i);
    if (ofs[i] < 0) return fail(SHT_ERR_INVALID_ARG, "ofs[%d] < 0", i);
    if (stride && stride[i] < 1) return fail(SHT_ERR_INVALID_ARG, "stride[%d] < 1", i);
    if (!isfinite(phi0[i])) return fail(SHT_ERR_INVALID_ARG, "phi0[%d] not finite", i);
    if (weight && !isfinite(weight[i])) return fail(SHT_ERR_INVALID_ARG, "weight[%d] not finite", i);
  }
  auto *g = new sht_geom_s;
  g->nrings = nrings;
  g->theta.assign(theta, theta + nrings);
  g->nphi.assign(nphi, nphi + nrings);
  g->phi0.assign(phi0, phi0 + nrings);
  g->ofs.assign(ofs, ofs + nrings);
  g->stride.assign(nrings, 1);
  if (stride) g->stride.assign(stride, stride + nrings);
  g->weight.assign(nrings, 1.0);
  if (weight) g->weight.assign(weight, weight + nrings);
  *out = g;
  return SHT_OK;
}

// Gauss-Legendre nodes by Newton's method in theta.  P_n(1 - u) is evaluated
// with the recursion written for u = 2 sin^2(theta/2) and the differences
// D_k = P_k - P_{k-1}, which stays accurate next to the poles; at a root the
// Gauss weight is 2 sin^2(theta) / (n P_{n-1})^2.
static void gl_eval(int n, long double th, long double *pn, long double *dn) {
  long double h = sinl(0.5L * th);
  long double u = 2.0L * h * h;
  long double p = 1.0L - u, d = -u;  // P_1, D_1
  if (n == 0) {
    *pn = 1.0L;
    *dn = 1.0L;
    return;
  }
  for (int k = 1; k < n; ++k) {
    d = (k * d - (2 * k + 1) * u * p) / (k + 1);
    p += d;
  }
  *pn = p;
  *dn = d;
}

static void gl_nodes(int n, std::vector<double> &th, std::vector<double> &w) {
  th.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    long double t = kPiL * (4 * i + 3) / (4 * n + 2);
    bool mid = (2 * i + 1 == n);
    if (mid) {
      t = 0.5L * kPiL;
    } else {
      for (int it = 0; it < 64; ++it) {
        long double pn, dn;
        gl_eval(n, t, &pn, &dn);
        long double h = sinl(0.5L * t);
        long double step = pn * sinl(t) / (n * (dn - 2.0L * h * h * pn));
        t -= step;
        if (fabsl(step) <= 1e-18L * t && it > 1) break;
      }
    }
    long double pn, dn;
    gl_eval(n, t, &pn, &dn);
    long double q = n * (pn - dn), s = sinl(t);
    double wi = (double)(2.0L * s * s / (q * q));
    th[i] = (double)t;
    w[i] = wi;
    th[n - 1 - i] = mid ? (double)t : (double)(kPiL - t);
    w[n - 1 - i] = wi;
  }
}

static int make_regular(const std::vector<double> &th, const std::vector<double> &wq, int nlon,
                        sht_geom_t *out) {
  int n = (int)th.size();
  std::vector<int> nphi(n, nlon);
  std::vector<double> phi0(n, 0.0), w(n);
  std::vector<int64_t> ofs(n);
  for (int i = 0; i < n; ++i) {
    ofs[i] = (int64_t)i * nlon;
    w[i] = wq[i] * 2.0 * M_PI / nlon;
  }
  return sht_geom_general(n, th.data(), nphi.data(), phi0.data(), ofs.data(), nullptr, w.data(), out);
}

// smallest n' >= n whose prime factors are 2, 3 and 5
static int smooth235(int n) {
  for (int k = std::max(n, 1);; ++k) {
    int r = k;
    for (int f : {2, 3, 5})
      while (r % f == 0) r /= f;
    if (r == 1) return k;
  }
}

// Sect. 4.4.2: Gauss-Legendre rings thinned by the polar optimisation.  Eq.
// eq_polaropt solved for m: sqrt(m^2 + s^2 - 2 m s cos(theta)) = T + lmax sin(theta).
// A ring carries the terms of both m and -m, for which the sign of m s cos(theta)
// differs, so its band limit is the larger root:
//   m_y = |s| |cos(theta)| + sqrt((T + lmax sin(theta))^2 - s^2 sin^2(theta)),
// T = max(100, 0.01 lmax), the same on mirrored rings (which thus keep sharing one
// Legendre evaluation); ring y gets the smallest 2^a 3^b 5^c >= 2 min(m_y, lmax) + 1
// pixels and the weight w_GL 2 pi / Nphi_y.
extern "C" int sht_geom_reduced_gauss(int nlat, int lmax, int spin, sht_geom_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nlat < 1 || lmax < 0) return fail(SHT_ERR_INVALID_ARG, "nlat >= 1 and lmax >= 0 required");
  std::vector<double> th, wq;
  gl_nodes(nlat, th, wq);
  const double T = std::max(100.0, 0.01 * lmax), s = std::abs(spin);
  std::vector<int> nphi(nlat);
  std::vector<double> phi0(nlat, 0.0), w(nlat);
  std::vector<int64_t> ofs(nlat);
  int64_t o = 0;
  for (int i = 0; i < nlat; ++i) {
    const double c = cos(th[i]), sn = sin(th[i]), r = T + lmax * sn;
    const double m = s * fabs(c) + sqrt(std::max(0.0, r * r - s * s * sn * sn));
    const int mm = (int)std::min<double>(lmax, floor(m));
    nphi[i] = smooth235(2 * mm + 1);
    ofs[i] = o;
    o += nphi[i];
    w[i] = wq[i] * 2.0 * M_PI / nphi[i];
  }
  return sht_geom_general(nlat, th.data(), nphi.data(), phi0.data(), ofs.data(), nullptr, w.data(), out);
}

extern "C" int sht_geom_gauss(int nlat, int nlon, sht_geom_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nlat < 1 || nlon < 1) return fail(SHT_ERR_INVALID_ARG, "nlat, nlon must be >= 1");
  std::vector<double> th, w;
  gl_nodes(nlat, th, w);
  return make_regular(th, w, nlon, out);
}

// ---- DFT of any length on the host, in long double ------------------------------
// X_i = sum_k x_k e^{+2 pi i k i / n}.  Bluestein's chirp identity turns it into a
// cyclic convolution, done with radix-2 transforms of a power-of-two length >= 2n - 1.
typedef std::complex<long double> cld;

static void fft2_ld(std::vector<cld> &a, bool inverse) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {  // bit reversal
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const long double ang = (inverse ? 2.0L : -2.0L) * kPiL / (long double)len;
    for (size_t k = 0; k < len / 2; ++k) {
      const cld w(cosl(ang * k), sinl(ang * k));
      for (size_t i = k; i < n; i += len) {
        const cld u = a[i], v = a[i + len / 2] * w;
        a[i] = u + v;
        a[i + len / 2] = u - v;
      }
    }
  }
}

static std::vector<cld> dft_pos_ld(const std::vector<cld> &x) {
  const int64_t n = (int64_t)x.size();
  if (n <= 64) {  // short: the sum itself
    std::vector<cld> X(n);
    for (int64_t i = 0; i < n; ++i) {
      cld s = 0;
      for (int64_t k = 0; k < n; ++k) {
        const long double ang = 2.0L * kPiL * (long double)((i * k) % n) / (long double)n;
        s += x[k] * cld(cosl(ang), sinl(ang));
      }
      X[i] = s;
    }
    return X;
  }
  // e^{2 pi i k i / n} = w_i w_k conj(w_{i-k}), w_j = e^{pi i j^2 / n} (j^2 reduced mod 2n)
  auto chirp = [&](int64_t j) {
    const int64_t q = (j * j) % (2 * n);
    const long double ang = kPiL * (long double)q / (long double)n;
    return cld(cosl(ang), sinl(ang));
  };
  size_t M = 1;
  while ((int64_t)M < 2 * n - 1) M <<= 1;
  std::vector<cld> a(M, 0), b(M, 0);
  for (int64_t k = 0; k < n; ++k) a[k] = x[k] * chirp(k);
  for (int64_t j = 0; j < n; ++j) {
    b[j] = std::conj(chirp(j));
    if (j) b[M - j] = b[j];
  }
  fft2_ld(a, false);
  fft2_ld(b, false);
  for (size_t i = 0; i < M; ++i) a[i] *= b[i];
  fft2_ld(a, true);
  std::vector<cld> X(n);
  for (int64_t i = 0; i < n; ++i) X[i] = chirp(i) * a[i] / (long double)M;
  return X;
}

// ECP colatitudes and quadrature weights on [-1, 1] (Fejer 1, Fejer 2,
// Clenshaw-Curtis; Sect. 4.4.1).  Each rule's weights are one DFT of the rule's
// moment sequence (Waldvogel 2006), so they cost O(n log n) instead of O(n^2):
//  CC, N = nlat - 1, theta_i = i pi / N:
//    w_i = (c_i / N) Re sum_k A_k e^{2 pi i k i / N}, A_0 = 1,
//    A_k = -b_k / (4k^2 - 1) for 1 <= k <= N/2 (b_k = 1 at k = N/2, else 2),
//    c_0 = c_N = 1, else 2 (w_N = w_0);
//  Fejer 1, N = nlat, theta_i = (i + 1/2) pi / N:
//    w_i = (2 / N) Re sum_k A_k e^{i pi k / N} e^{2 pi i k i / N}, A_0 = 1,
//    A_k = -2 / (4k^2 - 1) for 1 <= k <= N/2;
//  Fejer 2, N = nlat + 1, theta_i = i pi / N, i = 1..N-1:
//    w_i = (4 sin(theta_i) / N) Im[e^{-i pi i / N} sum_k S_k e^{2 pi i k i / N}],
//    S_k = 1 / (2k - 1) for 1 <= k <= N/2, since sin((2k-1) theta_i) is the
//    imaginary part of e^{-i pi i / N} e^{2 pi i k i / N}.
extern "C" int sht_geom_ecp(int kind, int nlat, int nlon, sht_geom_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nlat < 1 || nlon < 1) return fail(SHT_ERR_INVALID_ARG, "nlat, nlon must be >= 1");
  std::vector<double> th(nlat), w(nlat);
  if (kind == SHT_ECP_FEJER1) {
    const int N = nlat;
    std::vector<cld> A(N, 0);
    A[0] = 1;
    for (int k = 1; 2 * k <= N; ++k) {
      const long double ang = kPiL * k / N;
      A[k] = cld(cosl(ang), sinl(ang)) * (-2.0L / (4.0L * k * k - 1.0L));
    }
    const std::vector<cld> X = dft_pos_ld(A);
    for (int i = 0; i < N; ++i) {
      th[i] = (double)(kPiL * (2 * i + 1) / (2 * N));
      w[i] = (double)(X[i].real() * 2.0L / N);
    }
  } else if (kind == SHT_ECP_FEJER2) {
    const int N = nlat + 1;
    std::vector<cld> S(N, 0);
    for (int k = 1; 2 * k <= N; ++k) S[k] = 1.0L / (2 * k - 1);
    const std::vector<cld> X = dft_pos_ld(S);
    for (int i = 1; i < N; ++i) {
      const long double t = kPiL * i / N;
      const cld z = cld(cosl(t), -sinl(t)) * X[i];
      th[i - 1] = (double)t;
      w[i - 1] = (double)(4.0L * sinl(t) * z.imag() / N);
    }
  } else if (kind == SHT_ECP_CC) {
    if (nlat < 2) return fail(SHT_ERR_INVALID_ARG, "Clenshaw-Curtis needs nlat >= 2");
    const int N = nlat - 1;
    std::vector<cld> A(N, 0);
    A[0] = 1;
    for (int k = 1; 2 * k <= N; ++k) A[k] = -((2 * k == N) ? 1.0L : 2.0L) / (4.0L * k * k - 1.0L);
    const std::vector<cld> X = dft_pos_ld(A);
    for (int i = 0; i <= N; ++i) {
      th[i] = (double)(kPiL * i / N);
      w[i] = (double)(((i == 0 || i == N) ? 1.0L : 2.0L) * X[i % N].real() / N);
    }
  } else {
    return fail(SHT_ERR_INVALID_ARG, "unknown ECP kind %d", kind);
  }
  return make_regular(th, w, nlon, out);
}

extern "C" int sht_geom_healpix(int nside, sht_geom_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nside < 1 || nside > (1 << 20)) return fail(SHT_ERR_INVALID_ARG, "nside out of range");
  const int nr = 4 * nside - 1;
  std::vector<double> th(nr), p0(nr), w(nr, 4.0 * M_PI / (12.0 * (double)nside * nside));
  std::vector<int> np(nr);
  std::vector<int64_t> ofs(nr);
  int64_t o = 0;
  for (int r = 0; r < nr; ++r) {
    int i = r + 1;                                // ring number from the north pole
    int k = (i <= 2 * nside) ? i : 4 * nside - i;  // mirrored ring number
    long double t;
    if (k < nside) {  // polar cap: 1 - z = k^2 / (3 nside^2) = 2 sin^2(theta/2)
      t = 2.0L * asinl(k / (sqrtl(6.0L) * nside));
      np[r] = 4 * k;
      p0[r] = (double)(kPiL / (4 * k));
    } else {  // equatorial belt: z = 4/3 - 2k / (3 nside)
      t = acosl((4.0L * nside - 2.0L * k) / (3.0L * nside));
      np[r] = 4 * nside;
      p0[r] = ((k - nside) % 2 == 0) ? (double)(kPiL / (4 * nside)) : 0.0;
    }
    th[r] = (i <= 2 * nside) ? (double)t : (double)(kPiL - t);
    ofs[r] = o;
    o += np[r];
  }
  return sht_geom_general(nr, th.data(), np.data(), p0.data(), ofs.data(), nullptr, w.data(), out);
}

extern "C" int sht_geom_subset(sht_geom_t g, int nsel, const int *rings, sht_geom_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!g || nsel < 1 || !rings) return fail(SHT_ERR_INVALID_ARG, "bad subset arguments");
  std::vector<char> seen(g->nrings, 0);
  std::vector<double> th, p0, w;
  std::vector<int> np, st;
  std::vector<int64_t> ofs;
  for (int k = 0; k < nsel; ++k) {
    int r = rings[k];
    if (r < 0 || r >= g->nrings) return fail(SHT_ERR_INVALID_ARG, "ring %d out of range", r);
    if (seen[r]) return fail(SHT_ERR_INVALID_ARG, "ring %d listed twice", r);
    seen[r] = 1;
    th.push_back(g->theta[r]);
    p0.push_back(g->phi0[r]);
    w.push_back(g->weight[r]);
    np.push_back(g->nphi[r]);
    st.push_back(g->stride[r]);
    ofs.push_back(g->ofs[r]);
  }
  return sht_geom_general(nsel, th.data(), np.data(), p0.data(), ofs.data(), st.data(), w.data(), out);
}

extern "C" int sht_geom_info(sht_geom_t g, int *nrings, int64_t *npix, int *npairs);

extern "C" int sht_geom_rings(sht_geom_t g, double *theta, int *nphi, double *phi0, int64_t *ofs,
                              int *stride, double *weight) {
  if (!g) return fail(SHT_ERR_INVALID_ARG, "geometry is NULL");
  for (int i = 0; i < g->nrings; ++i) {
    if (theta) theta[i] = g->theta[i];
    if (nphi) nphi[i] = g->nphi[i];
    if (phi0) phi0[i] = g->phi0[i];
    if (ofs) ofs[i] = g->ofs[i];
    if (stride) stride[i] = g->stride[i];
    if (weight) weight[i] = g->weight[i];
  }
  return SHT_OK;
}

extern "C" void sht_geom_destroy(sht_geom_t g) { delete g; }

// Ring pairing: rings y, y' with theta_y' = pi - theta_y (to 1e-12) and the
// same nphi share one Legendre evaluation through the parity relation
// sLambda_lm(pi - theta) = (-1)^(l+m) (-s)Lambda_lm(theta).  Pairs are ordered
// from the poles towards the equator so that the polar cut removes a prefix.
static void pair_rings(const sht_geom_s *g, std::vector<int> &pn, std::vector<int> &ps) {
  std::vector<int> idx(g->nrings);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    return g->theta[a] < g->theta[b] || (g->theta[a] == g->theta[b] && a < b);
  });
  pn.clear();
  ps.clear();
  int i = 0, j = g->nrings - 1;
  while (i <= j) {
    int a = idx[i], b = idx[j];
    if (i == j) {
      pn.push_back(a);
      ps.push_back(-1);
      break;
    }
    double d = g->theta[a] + g->theta[b] - M_PI;
    if (fabs(d) <= 1e-12 && g->nphi[a] == g->nphi[b] && g->theta[a] < 0.5 * M_PI) {
      pn.push_back(a);
      ps.push_back(b);
      ++i;
      --j;
    } else if (d < 0) {  // ring a has no southern mirror
      pn.push_back(a);
      ps.push_back(-1);
      ++i;
    } else {
      pn.push_back(b);
      ps.push_back(-1);
      --j;
    }
  }
  // order by distance from the nearest pole
  std::vector<int> ord(pn.size());
  std::iota(ord.begin(), ord.end(), 0);
  auto pd = [&](int k) { double t = g->theta[pn[k]]; return std::min(t, M_PI - t); };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return pd(a) < pd(b); });
  std::vector<int> pn2, ps2;
  for (int k : ord) {
    pn2.push_back(pn[k]);
    ps2.push_back(ps[k]);
  }
  pn.swap(pn2);
  ps.swap(ps2);
}

extern "C" int sht_geom_info(sht_geom_t g, int *nrings, int64_t *npix, int *npairs) {
  if (!g) return fail(SHT_ERR_INVALID_ARG, "geometry is NULL");
  if (nrings) *nrings = g->nrings;
  if (npix) {
    int64_t mx = 0;
    for (int i = 0; i < g->nrings; ++i)
      mx = std::max<int64_t>(mx, g->ofs[i] + (int64_t)(g->nphi[i] - 1) * g->stride[i] + 1);
    *npix = mx;
  }
  if (npairs) {
    std::vector<int> pn, ps;
    pair_rings(g, pn, ps);
    *npairs = (int)pn.size();
  }
  return SHT_OK;
}

// ----------------------------------------------------------------------------
// a_lm layout
// ----------------------------------------------------------------------------
extern "C" int sht_alm_create(int lmax, int mmax, int nm, const int *mval, const int64_t *mstart,
                              int stride, sht_alm_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (lmax < 0 || mmax < 0 || mmax > lmax || lmax > 65535)
    return fail(SHT_ERR_INVALID_ARG, "need 0 <= mmax <= lmax <= 65535");
  if (stride < 1) return fail(SHT_ERR_INVALID_ARG, "stride < 1");
  auto *a = new sht_alm_s;
  a->lmax = lmax;
  a->mmax = mmax;
  a->stride = stride;
  if (!mval) {
    a->nm = mmax + 1;
    for (int m = 0; m <= mmax; ++m) a->mval.push_back(m);
  } else {
    if (nm < 1 || nm > mmax + 1) {
      delete a;
      return fail(SHT_ERR_INVALID_ARG, "nm out of range");
    }
    std::vector<char> seen(mmax + 1, 0);
    for (int i = 0; i < nm; ++i) {
      if (mval[i] < 0 || mval[i] > mmax || seen[mval[i]]) {
        delete a;
        return fail(SHT_ERR_INVALID_ARG, "mval[%d] invalid or repeated", i);
      }
      seen[mval[i]] = 1;
      a->mval.push_back(mval[i]);
    }
    a->nm = nm;
  }
  if (mstart) {
    for (int i = 0; i < a->nm; ++i) {
      if (mstart[i] + (int64_t)a->mval[i] * stride < 0) {
        delete a;
        return fail(SHT_ERR_INVALID_ARG, "mstart[%d] gives a negative index", i);
      }
      a->mstart.push_back(mstart[i]);
    }
  } else {
    // triangular m-major over the listed m: entries l = m..lmax follow each other
    int64_t o = 0;
    for (int i = 0; i < a->nm; ++i) {
      int m = a->mval[i];
      a->mstart.push_back(o - (int64_t)m * stride);
      o += (int64_t)(lmax + 1 - m) * stride;
    }
  }
  *out = a;
  return SHT_OK;
}

extern "C" int sht_alm_size(sht_alm_t a, int64_t *n) {
  if (!a || !n) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  int64_t mx = 0;
  for (int i = 0; i < a->nm; ++i)
    mx = std::max<int64_t>(mx, a->mstart[i] + (int64_t)a->lmax * a->stride + 1);
  *n = mx;
  return SHT_OK;
}

extern "C" void sht_alm_destroy(sht_alm_t a) { delete a; }

// ----------------------------------------------------------------------------
// FFT planning (lengths, factorisations, Rader / Bluestein tables)
// ----------------------------------------------------------------------------
static bool factor_small(int n, std::vector<int> &rad) {
  rad.clear();
  while (n % 4 == 0) {
    rad.push_back(4);
    n /= 4;
  }
  if (n % 2 == 0) {
    rad.push_back(2);
    n /= 2;
  }
  for (int p = 3; p <= kMaxBigRadix && n > 1; p += 2) {
    while (n % p == 0) {
      rad.push_back(p);
      n /= p;
    }
  }
  return n == 1 && rad.size() <= 24;
}

// FP64 instructions per point of the passes rad (a model for choosing the
// Bluestein length): radix 2 and 4 cost 2 and 4 adds a point; an odd radix with
// h = (R-1)/2 costs 4 h^2 multiply-adds and 10 h adds a butterfly; every pass
// but the last adds a complex twiddle product (4 instructions) a point.
static double fft_cost_per_point(const std::vector<int> &rad) {
  double c = 0.0;
  for (size_t i = 0; i < rad.size(); ++i) {
    const int R = rad[i];
    if (R == 2 || R == 4) {
      c += R;
    } else {
      const double h = (R - 1) / 2;
      c += (4.0 * h * h + 10.0 * h) / R;
    }
    if (i + 1 < rad.size()) c += 4.0;
  }
  return c;
}

static bool is_prime(int n) {
  if (n < 2) return false;
  for (int d = 2; (int64_t)d * d <= n; ++d)
    if (n % d == 0) return false;
  return true;
}

static int64_t powmod(int64_t b, int64_t e, int64_t m) {
  int64_t r = 1;
  b %= m;
  while (e > 0) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return r;
}

static int primitive_root(int p) {
  std::vector<int> qs;
  int n = p - 1;
  for (int d = 2; (int64_t)d * d <= n; ++d)
    if (n % d == 0) {
      qs.push_back(d);
      while (n % d == 0) n /= d;
    }
  if (n > 1) qs.push_back(n);
  for (int g = 2; g < p; ++g) {
    bool ok = true;
    for (int q : qs)
      if (powmod(g, (p - 1) / q, p) == 1) {
        ok = false;
        break;
      }
    if (ok) return g;
  }
  return -1;
}

template <class T>
static int dev_upload(sht_plan_s *P, const std::vector<T> &h, const T **d) {
  void *ptr = nullptr;
  CUDA_TRY(cudaMalloc(&ptr, std::max<size_t>(1, h.size() * sizeof(T))));
  P->fft_allocs.push_back(ptr);
  P->workspace += h.size() * sizeof(T);
  if (!h.empty()) CUDA_TRY(cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  *d = (const T *)ptr;
  return SHT_OK;
}

static std::vector<double2> twiddles(int len) {
  std::vector<double2> w(len);
  for (int k = 0; k < len; ++k) {
    long double a = -2.0L * kPiL * k / len;
    w[k] = make_double2((double)cosl(a), (double)sinl(a));
  }
  return w;
}

// e^{-2 pi i k / len} as hi/lo float pairs, from long double
static std::vector<float4> twiddles_f(int len) {
  std::vector<float4> w(len);
  for (int k = 0; k < len; ++k) {
    const long double a = -2.0L * kPiL * k / len, c = cosl(a), s = sinl(a);
    w[k] = make_float4((float)c, (float)(c - (float)c), (float)s, (float)(s - (float)s));
  }
  return w;
}

// an FP64 table on the device as hi/lo float pairs (the double-float engine's copy)
static int upload_pairs(sht_plan_s *P, const double2 *d, int len, const float4 **out) {
  std::vector<double2> h(len);
  CUDA_TRY(cudaMemcpy(h.data(), d, len * sizeof(double2), cudaMemcpyDeviceToHost));
  std::vector<float4> f(len);
  for (int i = 0; i < len; ++i) {
    const float rh = (float)h[i].x, ih = (float)h[i].y;
    f[i] = make_float4(rh, (float)(h[i].x - (double)rh), ih, (float)(h[i].y - (double)ih));
  }
  return dev_upload(P, f, out);
}

// How a ring of n points is transformed (host logic only): kind 0 mixed radix
// of length n, 1 Rader (n prime, n-1 smooth) of length n-1, 2 Bluestein of the
// convolution length >= 2n-1 that the pass model rates cheapest among the
// smooth lengths up to the first one whose radices are all <= 31.  Returns
// false when no length up to kFftMaxGlobalLen fits.
static bool fft_choose(int n, int &kind, int &len, std::vector<int> &rad) {
  if (n <= kFftMaxGlobalLen && factor_small(n, rad)) {
    kind = 0;
    len = n;
    return true;
  }
  if (is_prime(n) && n - 1 <= kFftMaxGlobalLen && factor_small(n - 1, rad)) {
    kind = 1;
    len = n - 1;
    return true;
  }
  int best = 0;
  double best_cost = 0.0;
  for (int M = 2 * n - 1; M <= kFftMaxGlobalLen; ++M) {
    if (!factor_small(M, rad)) continue;
    const double c = M * fft_cost_per_point(rad);
    if (best == 0 || c < best_cost) {
      best = M;
      best_cost = c;
    }
    if (rad.back() <= kMaxRadix) break;
  }
  if (best == 0) return false;
  factor_small(best, rad);
  kind = 2;
  len = best;
  return true;
}

extern "C" int sht_fft_plan_info(int n, int *kind, int *len, int *nrad, int *radices) {
  if (!kind || !len || !nrad || !radices) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(SHT_ERR_INVALID_ARG, "ring length must be >= 1");
  std::vector<int> rad;
  if (!fft_choose(n, *kind, *len, rad))
    return fail(SHT_ERR_UNSUPPORTED, "ring length %d: no FFT of size <= %d available", n, kFftMaxGlobalLen);
  *nrad = (int)rad.size();
  for (int i = 0; i < *nrad; ++i) radices[i] = rad[i];
  return SHT_OK;
}

static int build_fft_plan(sht_plan_s *P, int n, FftPlanDev &fp, FftPlanDev *scratch_dev) {
  memset(&fp, 0, sizeof(fp));
  fp.n = n;
  std::vector<int> rad;
  int rc;
  if (!fft_choose(n, fp.kind, fp.len, rad))
    return fail(SHT_ERR_UNSUPPORTED, "ring length %d: no FFT of size <= %d available", n, kFftMaxGlobalLen);
  fp.nrad = (int)rad.size();
  for (int i = 0; i < fp.nrad; ++i) fp.rad[i] = rad[i];
  if ((rc = dev_upload(P, twiddles(fp.len), &fp.w)) != SHT_OK) return rc;
  if (fp.kind == 0) {  // X_k ends at sum_i (k_i) len / (R_0 ... R_i), k = k_0 + R_0 (k_1 + R_1 (...))
    std::vector<int> pos(n);
    for (int k = 0; k < n; ++k) {
      int kk = k, L = n, at = 0;
      for (int r : rad) {
        L /= r;
        at += (kk % r) * L;
        kk /= r;
      }
      pos[k] = at;
    }
    if ((rc = dev_upload(P, pos, &fp.pos)) != SHT_OK) return rc;
  }

  if (fp.kind == 1) {
    const int g = primitive_root(n);
    const int L = n - 1;
    std::vector<int> pin(L), inv(n, 0);
    int64_t ginv = powmod(g, n - 2, n);
    int64_t a = 1, b = 1;
    std::vector<double2> kern(L);
    for (int q = 0; q < L; ++q) {
      pin[q] = (int)a;     // g^q
      inv[b] = q;          // g^{-q} = b
      long double ang = -2.0L * kPiL * (long double)b / n;
      kern[q] = make_double2((double)cosl(ang), (double)sinl(ang));
      a = a * g % n;
      b = b * ginv % n;
    }
    if ((rc = dev_upload(P, pin, &fp.perm_in)) != SHT_OK) return rc;
    if ((rc = dev_upload(P, inv, &fp.inv_out)) != SHT_OK) return rc;
    const double2 *dk;
    if ((rc = dev_upload(P, kern, &dk)) != SHT_OK) return rc;
    std::vector<double2> zero(L);
    const double2 *ds;
    if ((rc = dev_upload(P, zero, &ds)) != SHT_OK) return rc;
    fp.spec = ds;
    CUDA_TRY(cudaMemcpy(scratch_dev, &fp, sizeof(fp), cudaMemcpyHostToDevice));
    CUDA_TRY(launch_fft_spectrum(&fp, scratch_dev, dk, (double2 *)ds, L, 1.0 / L, 0));
    CUDA_TRY(cudaDeviceSynchronize());
  } else if (fp.kind == 2) {
    const int M = fp.len;
    std::vector<double2> chirp(n), h(M, make_double2(0.0, 0.0));
    for (int k = 0; k < n; ++k) {
      int64_t q = ((int64_t)k * k) % (2 * (int64_t)n);  // e^{-pi i k^2 / n} depends on k^2 mod 2n
      long double ang = -kPiL * (long double)q / n;
      chirp[k] = make_double2((double)cosl(ang), (double)sinl(ang));
      double2 c = make_double2(chirp[k].x, -chirp[k].y);
      h[k] = c;
      if (k > 0) h[M - k] = c;
    }
    if ((rc = dev_upload(P, chirp, &fp.chirp)) != SHT_OK) return rc;
    const double2 *dh;
    if ((rc = dev_upload(P, h, &dh)) != SHT_OK) return rc;
    std::vector<double2> zero(M);
    const double2 *ds;
    if ((rc = dev_upload(P, zero, &ds)) != SHT_OK) return rc;
    fp.spec = ds;
    CUDA_TRY(cudaMemcpy(scratch_dev, &fp, sizeof(fp), cudaMemcpyHostToDevice));
    CUDA_TRY(launch_fft_spectrum(&fp, scratch_dev, dh, (double2 *)ds, M, 1.0 / M, 0));
    CUDA_TRY(cudaDeviceSynchronize());
  }
  if (P->precision == SHT_MIXED) {  // the double-float engine's tables
    if ((rc = dev_upload(P, twiddles_f(fp.len), &fp.wf)) != SHT_OK) return rc;
    if (fp.kind != 0 && (rc = upload_pairs(P, fp.spec, fp.len, &fp.specf)) != SHT_OK) return rc;
    if (fp.kind == 2 && (rc = upload_pairs(P, fp.chirp, n, &fp.chirpf)) != SHT_OK) return rc;
  }
  return SHT_OK;
}

// Polar cut (Sect. 3.3): skip (m, pair) when
//   sqrt(m^2 + s^2 - 2 m s cos theta) - lmax sin theta > T,  T = max(100, 0.01 lmax),
// for both rings of the pair (cos theta and -cos theta: the smaller root, |m s| |cos theta|).
// Pairs run from the poles towards the equator, so for each m the cut is a
// prefix: the result is the index of the first pair kept (npairs if none).
static std::vector<int> polar_first_pairs(const sht_geom_s *g, const std::vector<int> &pair_n, int lmax, int spin,
                                          const std::vector<int> &mval) {
  const double T = std::max(100.0, 0.01 * lmax), s = spin;
  const int npairs = (int)pair_n.size();
  std::vector<int> first(mval.size(), npairs);
  for (size_t i = 0; i < mval.size(); ++i) {
    const double m = mval[i];
    for (int p = 0; p < npairs; ++p) {
      const double th = g->theta[pair_n[p]];
      const double c = fabs(cos(th)), sn = sin(th);
      const double v = sqrt(std::max(0.0, m * m + s * s - 2.0 * fabs(m * s) * c)) - lmax * sn;
      if (!(v > T)) {
        first[i] = p;
        break;
      }
    }
  }
  return first;
}

extern "C" int sht_geom_polar_cut(sht_geom_t g, int lmax, int spin, int nm, const int *mval, int *first_pair,
                                  double *pair_theta, int64_t *triples) {
  if (!g || !mval || !first_pair || !triples) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  if (lmax < 0 || nm < 1) return fail(SHT_ERR_INVALID_ARG, "lmax >= 0 and nm >= 1 required");
  std::vector<int> pn, ps;
  pair_rings(g, pn, ps);
  std::vector<int> mv(mval, mval + nm);
  for (int m : mv)
    if (m < 0 || m > lmax) return fail(SHT_ERR_INVALID_ARG, "m = %d outside 0..lmax", m);
  const std::vector<int> first = polar_first_pairs(g, pn, lmax, spin, mv);
  const int as = spin < 0 ? -spin : spin;
  int64_t trip = 0;
  for (int i = 0; i < nm; ++i) {
    first_pair[i] = first[i];
    const int nl = lmax - std::max(mv[i], as) + 1;
    if (nl > 0) trip += (int64_t)(pn.size() - first[i]) * nl;
  }
  if (pair_theta)
    for (size_t p = 0; p < pn.size(); ++p) pair_theta[p] = g->theta[pn[p]];
  *triples = trip;
  return SHT_OK;
}

// ----------------------------------------------------------------------------
// Plans
// ----------------------------------------------------------------------------
static void free_plan(sht_plan_s *P) {
  if (!P) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(P->device);
  void *ptrs[] = {P->d_pairs, P->d_pair_rings, P->d_rings, P->d_mval, P->d_mstart, P->d_coef_off,
                  P->d_coef, P->d_coef32, P->d_alm32, P->d_pm64, P->d_mpre, P->d_minv, P->d_phase, P->d_part, P->d_fft,
                  P->d_pair_fft, P->d_fft_scratch, P->d_err, P->d_join};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 2; ++k) {
    if (P->d_syn_items[k]) cudaFree(P->d_syn_items[k]);
    if (P->d_syn_first[k]) cudaFree(P->d_syn_first[k]);
    if (P->d_ana_items[k]) cudaFree(P->d_ana_items[k]);
    if (P->d_ana_part_off[k]) cudaFree(P->d_ana_part_off[k]);
    if (P->d_ana_nslot[k]) cudaFree(P->d_ana_nslot[k]);
    if (P->d_syn_lo[k]) cudaFree(P->d_syn_lo[k]);
    if (P->d_ana_lo[k]) cudaFree(P->d_ana_lo[k]);
  }
  for (void *p : P->fft_allocs) cudaFree(p);
  if (P->side) cudaStreamDestroy(P->side);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->ev_lo) cudaEventDestroy(P->ev_lo);
  for (auto &r : P->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (cur >= 0) cudaSetDevice(cur);
  delete P;
}

template <class T>
static int upload(sht_plan_s *P, const std::vector<T> &h, T **d) {
  CUDA_TRY(cudaMalloc((void **)d, std::max<size_t>(1, h.size() * sizeof(T))));
  P->workspace += h.size() * sizeof(T);
  if (!h.empty()) CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SHT_OK;
}

// Tilings of the analysis Legendre kernels (ring pairs per thread) built for a
// spin class and padded job count; the first is the default.
static std::vector<int> ana_ppt_candidates(int spin, int nj) {
  if (spin == 0) {
    if (nj == 1) return {4, 8, 2};
    if (nj == 2) return {4, 2};
    return {2};
  }
  if (nj == 1) return {2, 4, 1};
  if (nj == 2) return {2, 1};
  return {2};
}

// Mixed form: columns m below this run in FP64 on the rings near the poles.  The
// double-float recursion keeps ~48 bits; for small m near the poles it is
// non-oscillatory over l < ~m/theta, where its per-step rounding grows like a
// power of l.  On the rings nearest a pole the columns m > |s| still carry
// weight theta^(m-|s|), so enough of them must run in FP64 for each ring's own
// error (not only the map's) to stay below 1e-10: lmax / 170 columns (12 at
// lmax 2047, 24 at 4095, 48 at 8191) keep every ring near or below 5e-11 in
// spin-2 synthesis (measured against the FP64 form ring by ring), and their
// FP64 items stay hidden on the side stream.  Below lmax 2000 the rings' errors
// are below 3e-11 without them, and the items would no longer be hidden.
static int default_fp64_columns(int lmax) { return lmax < 2000 ? 0 : lmax / 170; }

// Entries of the coefficient table that the columns m < m_below occupy, as a
// prefix (their last entry + 1): what a mixed plan's FP64 tables must hold.
static int64_t fp64_prefix(const sht_plan_s *P, int m_below) {
  int64_t n = 0;
  for (int i = 0; i < P->nm; ++i)
    if (P->mval[i] < m_below) {
      const int l0 = std::max(P->mval[i], std::abs(P->spin));
      n = std::max<int64_t>(n, P->coef_off[i] + std::max(0, P->lmax - l0 + 1));
    }
  return n;
}

// an item of column mi over ring pairs [p0, p1) runs in FP64 (mixed plans only)
static bool lo_item(const sht_plan_s *P, int mi, int p0, int p1) {
  if (P->precision != SHT_MIXED || P->mval[mi] >= P->fp64_m_below) return false;
  for (int p = p0; p < p1 && p < P->npairs; ++p)
    if (P->pair_pole[p] < kFp64PolarCap) return true;
  return false;
}

template <class T>
static int upload_list(sht_plan_s *P, const std::vector<std::pair<int64_t, T>> &list, T **d, int *n) {
  std::vector<T> v;
  for (auto &e : list) v.push_back(e.second);
  if (*d) cudaFree(*d);
  *d = nullptr;
  *n = (int)v.size();
  return upload(P, v, d);
}

// Synthesis work lists: per polar variant the cost-sorted (m, first pair)
// tiles (the mixed form's FP64 columns in lists of their own), each m's first
// synthesised pair, and the exact triple count.
static int build_syn_lists(sht_plan_s *P) {
  int rc;
  const int as = abs(P->spin);
  for (int polar = 0; polar < 2; ++polar) {
    std::vector<std::pair<int64_t, int2>> syn, lo;
    std::vector<int> sfirst(P->nm);
    int64_t trip = 0;
    for (int i = 0; i < P->nm; ++i) {
      int l0 = std::max(P->mval[i], as);
      int nl = P->lmax - l0 + 1;
      if (nl <= 0) {
        sfirst[i] = P->npairs;
        continue;
      }
      int fp = polar ? P->first_pair[i] : 0;
      trip += (int64_t)(P->npairs - fp) * nl;
      int sf = (fp / kSynTile) * kSynTile;
      sfirst[i] = sf;
      for (int p = sf; p < P->npairs; p += kSynTile)
        (lo_item(P, i, p, p + kSynTile) ? lo : syn)
            .push_back({(int64_t)nl * std::min(kSynTile, P->npairs - p), make_int2(i, p)});
    }
    P->triples[polar] = trip;
    std::stable_sort(syn.begin(), syn.end(), [](auto &a, auto &b) { return a.first > b.first; });
    std::stable_sort(lo.begin(), lo.end(), [](auto &a, auto &b) { return a.first > b.first; });
    P->syn_list[polar] = syn;
    P->syn_list_lo[polar] = lo;
    if ((rc = upload_list(P, syn, &P->d_syn_items[polar], &P->nsyn_items[polar])) != SHT_OK) return rc;
    if ((rc = upload_list(P, lo, &P->d_syn_lo[polar], &P->nsyn_lo[polar])) != SHT_OK) return rc;
    if (P->d_syn_first[polar]) cudaFree(P->d_syn_first[polar]);
    P->d_syn_first[polar] = nullptr;
    if ((rc = upload(P, sfirst, &P->d_syn_first[polar])) != SHT_OK) return rc;
  }
  return SHT_OK;
}

// Analysis work lists: per polar variant the cost-sorted items and, per m, where
// their partial sums go.  A tile is kAnaThreads * ppt ring pairs; a mixed-form item
// walks a group of consecutive tiles of one m one after another and sums them into
// one slot of partial sums, so the partials' size shrinks by the group size (their
// DRAM traffic only while the slots of the resident CTAs fit in L2).  Groups are
// as large as keeps at least kAnaItemsPerSm items per SM (and at most
// kAnaGroupTiles tiles): the same work in fewer, longer CTAs, which on
// GB300 at lmax 4095 is as fast as one CTA per tile (152.5 against 153.0 ms per
// pair) with a sixteenth of the partials; an 8-map plan's analysis kernel is 4.4
// ms slower grouped, its slot reduction 6.6 ms faster (lmax 4095: 157.3 + 1.1
// against 152.9 + 7.7 ms).  FP64 items (the FP64 form, and a mixed plan's tiles
// next to the poles) take one tile each.  Item (m index, first tile,
// slot << 8 | tiles, -); the slots of m are summed by the reduction kernel.
static int build_ana_lists(sht_plan_s *P, int ppt) {
  int rc;
  const int as = abs(P->spin);
  const int V = (P->spin ? 4 : 2) * P->njobs_pad;  // doubles per l in the analysis partials
  const int TA = kAnaThreads * ppt;
  const int tiles = (P->npairs + TA - 1) / TA;
  const bool mixed = P->precision == SHT_MIXED;
  int group = 1;
  if (mixed) {  // tiles of the polar-cut variant (the default) over items per SM wanted
    int64_t ntile = 0;
    for (int i = 0; i < P->nm; ++i)
      if (P->lmax >= std::max(P->mval[i], as)) ntile += tiles - P->first_pair[i] / TA;
    group = (int)std::max<int64_t>(1, std::min<int64_t>(kAnaGroupTiles, ntile / ((int64_t)kAnaItemsPerSm * P->sms)));
  }
  int64_t need = 0;
  for (int polar = 0; polar < 2; ++polar) {
    std::vector<std::pair<int64_t, int4>> ana, lo;
    std::vector<int64_t> poff(P->nm);
    std::vector<int> nslot(P->nm, 0);
    int64_t off = 0;
    for (int i = 0; i < P->nm; ++i) {
      int l0 = std::max(P->mval[i], as);
      int nl = P->lmax - l0 + 1;
      poff[i] = off;
      if (nl <= 0) continue;
      int fp = polar ? P->first_pair[i] : 0;
      int slot = 0;
      for (int t = fp / TA; t < tiles;) {
        const auto cost = [&](int tt) { return (int64_t)nl * std::min(TA, P->npairs - tt * TA); };
        if (lo_item(P, i, t * TA, (t + 1) * TA)) {
          lo.push_back({cost(t), make_int4(i, t, (slot << 8) | 1, 0)});
          ++t;
        } else {
          int n = 0;
          int64_t c = 0;
          while (n < group && t + n < tiles && !lo_item(P, i, (t + n) * TA, (t + n + 1) * TA)) c += cost(t + n++);
          ana.push_back({c, make_int4(i, t, (slot << 8) | n, 0)});
          t += n;
        }
        ++slot;
      }
      nslot[i] = slot;
      off += (int64_t)slot * nl * V;
    }
    std::stable_sort(ana.begin(), ana.end(), [](auto &a, auto &b) { return a.first > b.first; });
    std::stable_sort(lo.begin(), lo.end(), [](auto &a, auto &b) { return a.first > b.first; });
    if (P->d_ana_part_off[polar]) cudaFree(P->d_ana_part_off[polar]);
    if (P->d_ana_nslot[polar]) cudaFree(P->d_ana_nslot[polar]);
    P->d_ana_part_off[polar] = nullptr;
    P->d_ana_nslot[polar] = nullptr;
    P->ana_list[polar] = ana;
    P->ana_list_lo[polar] = lo;
    if ((rc = upload_list(P, ana, &P->d_ana_items[polar], &P->nana_items[polar])) != SHT_OK) return rc;
    if ((rc = upload_list(P, lo, &P->d_ana_lo[polar], &P->nana_lo[polar])) != SHT_OK) return rc;
    if ((rc = upload(P, poff, &P->d_ana_part_off[polar])) != SHT_OK) return rc;
    if ((rc = upload(P, nslot, &P->d_ana_nslot[polar])) != SHT_OK) return rc;
    need = std::max(need, off);
  }
  if (need != P->part_doubles || !P->d_part) {  // sized for the current tiling
    if (P->d_part) cudaFree(P->d_part);
    P->d_part = nullptr;
    P->workspace += (need - P->part_doubles) * (int64_t)sizeof(double);
    P->part_doubles = need;
    CUDA_TRY(cudaMalloc(&P->d_part, std::max<int64_t>(1, P->part_doubles) * sizeof(double)));
  }
  P->ana_ppt = ppt;
  return SHT_OK;
}

static int plan_build(sht_plan_s *P, const sht_geom_s *g) {
  int rc;
  // ---- ring pairs ----
  pair_rings(g, P->pair_n, P->pair_s);
  P->npairs = (int)P->pair_n.size();
  P->nrings = g->nrings;
  std::vector<PairDev> pd(P->npairs);
  std::vector<int2> pr(P->npairs);
  P->pair_pole.resize(P->npairs);
  for (int p = 0; p < P->npairs; ++p) {
    double th = g->theta[P->pair_n[p]];
    P->pair_pole[p] = std::min(th, (double)kPiL - th);
    long double t = th;
    PairDev &d = pd[p];
    d.x = cos(th);
    long double sn = sinl(t), tn = tanl(0.5L * t);
    long double l1 = (sn > 0) ? log2l(sn) : 0.0L, l2 = (tn > 0) ? log2l(tn) : 0.0L;
    d.l1_hi = (double)l1;
    d.l1_lo = (double)(l1 - (long double)d.l1_hi);
    d.l2_hi = (double)l2;
    d.l2_lo = (double)(l2 - (long double)d.l2_hi);
    d.pole = (th == 0.0 || th == M_PI) ? 1 : 0;
    d.south = P->pair_s[p] >= 0;
    pr[p] = make_int2(P->pair_n[p], P->pair_s[p]);
  }
  if ((rc = upload(P, pd, &P->d_pairs)) != SHT_OK) return rc;
  if ((rc = upload(P, pr, &P->d_pair_rings)) != SHT_OK) return rc;
  std::vector<RingDev> rd(g->nrings);
  for (int r = 0; r < g->nrings; ++r) {
    rd[r].ofs = g->ofs[r];
    rd[r].nphi = g->nphi[r];
    rd[r].stride = g->stride[r];
    rd[r].phi0 = g->phi0[r];
    rd[r].weight = g->weight[r];
  }
  if ((rc = upload(P, rd, &P->d_rings)) != SHT_OK) return rc;

  // ---- m list and coefficient table layout ----
  const int as = abs(P->spin);
  std::vector<int64_t> coff(P->nm);
  int64_t nco = 0;
  for (int i = 0; i < P->nm; ++i) {
    int l0 = std::max(P->mval[i], as);
    coff[i] = nco;
    nco += std::max(0, P->lmax - l0 + 1);
  }
  P->coef_off = coff;
  P->ncoef = nco;
  std::vector<int> minv(P->mmax + 1, -1);
  for (int i = 0; i < P->nm; ++i) minv[P->mval[i]] = i;
  P->m_identity = 1;
  for (int i = 0; i < P->nm; ++i) P->m_identity &= P->mval[i] == i;
  if ((rc = upload(P, P->mval, &P->d_mval)) != SHT_OK) return rc;
  if ((rc = upload(P, P->mstart, &P->d_mstart)) != SHT_OK) return rc;
  if ((rc = upload(P, coff, &P->d_coef_off)) != SHT_OK) return rc;
  if ((rc = upload(P, minv, &P->d_minv)) != SHT_OK) return rc;
  // the FP64 tables: every entry for an FP64 plan; for a mixed plan the prefix its
  // default FP64 columns read (grown by sht_plan_set_fp64_columns when needed)
  P->ncoef64 = P->precision == SHT_MIXED ? fp64_prefix(P, default_fp64_columns(P->lmax)) : nco;
  CUDA_TRY(cudaMalloc(&P->d_coef, std::max<int64_t>(1, P->ncoef64) * sizeof(Coef)));
  P->workspace += P->ncoef64 * sizeof(Coef);
  if (P->precision == SHT_MIXED) {
    CUDA_TRY(cudaMalloc(&P->d_coef32, std::max<int64_t>(1, nco) * 2 * sizeof(float4)));
    P->workspace += nco * 2 * sizeof(float4);
    CUDA_TRY(cudaMalloc(&P->d_alm32, std::max<int64_t>(1, nco) * P->nmaps_pad * sizeof(float4)));
    P->workspace += nco * P->nmaps_pad * sizeof(float4);
  }
  if (P->spin != 0 && (P->precision == SHT_FP64 || default_fp64_columns(P->lmax) > 0)) {
    CUDA_TRY(cudaMalloc(&P->d_pm64, std::max<int64_t>(1, P->ncoef64) * P->nmaps_pad * sizeof(double2)));
    P->workspace += P->ncoef64 * P->nmaps_pad * sizeof(double2);
  }
  CUDA_TRY(cudaMalloc(&P->d_mpre, P->nm * sizeof(double2)));
  CUDA_TRY(cudaMalloc(&P->d_err, sizeof(int)));
  CUDA_TRY(cudaMemset(P->d_err, 0, sizeof(int)));
  if (P->precision == SHT_MIXED) {
    P->tc_lam_bound = tc_lambda_bound(P->lmax);
    CUDA_TRY(tc_prepare_device());
    CUDA_TRY(tc_ana_prepare_device());
    // the tensor-core synthesis by default wherever it was measured faster: every
    // supported shape except a single spin-0 map (lmax 4095: 32.1 ms against 25.6)
    P->tc_syn = tc_supported(P->spin, P->njobs_pad) && !(P->spin == 0 && P->njobs_pad == 1);
  }
  CUDA_TRY(launch_coef_tables(P, 0));
  if (P->precision == SHT_MIXED && P->nm > 0 && P->npairs > 0) {
    // where each ring pair's terms start, per m (the mixed Legendre kernels skip
    // the recursion over the negligible stretch before it)
    const size_t bytes = (size_t)P->nm * P->npairs * 3 * sizeof(float4);
    CUDA_TRY(cudaMalloc(&P->d_join, bytes));
    P->workspace += bytes;
    CUDA_TRY(launch_join_records(P, 0));
  }
  CUDA_TRY(cudaDeviceSynchronize());

  P->first_pair = polar_first_pairs(g, P->pair_n, P->lmax, P->spin, P->mval);
  if (P->d_join) {  // the steps left after the join records, over the pairs the polar cut keeps
    std::vector<int> lj((size_t)P->nm * P->npairs);
    CUDA_TRY(cudaMemcpy2D(lj.data(), sizeof(int), reinterpret_cast<const char *>(P->d_join) + 2 * sizeof(float4) + 8,
                          3 * sizeof(float4), sizeof(int), lj.size(), cudaMemcpyDeviceToHost));
    int64_t t = 0;
    for (int i = 0; i < P->nm; ++i)
      for (int p = P->first_pair[i]; p < P->npairs; ++p) {
        const int l = lj[(size_t)i * P->npairs + p];
        if (l <= P->lmax) t += P->lmax - l + 1;
      }
    P->triples_joined = t;
  }

  // ---- work lists ----
  P->fp64_m_below = P->precision == SHT_MIXED ? default_fp64_columns(P->lmax) : 0;
  if (P->precision == SHT_MIXED) {
    // high priority: the few long FP64 CTAs should start among the first, not
    // after the thousands of mixed CTAs queued beside them
    int least = 0, greatest = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CUDA_TRY(cudaStreamCreateWithPriority(&P->side, cudaStreamNonBlocking, greatest));
    for (cudaEvent_t *ev : {&P->ev_fork, &P->ev_join, &P->ev_lo})
      CUDA_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  }
  if ((rc = build_syn_lists(P)) != SHT_OK) return rc;
  if ((rc = build_ana_lists(P, ana_ppt_candidates(P->spin, P->njobs_pad)[0])) != SHT_OK) return rc;

  // ---- phase-array workspace F/G [nmaps][nm][npairs][2] ----
  size_t nph = (size_t)P->nmaps_pad * P->nm * P->npairs * 2;
  CUDA_TRY(cudaMalloc(&P->d_phase, std::max<size_t>(1, nph) * sizeof(double2)));
  P->workspace += nph * sizeof(double2);

  // ---- FFT plans per distinct ring length ----
  std::map<int, int> lens;
  std::vector<int> pf(P->npairs);
  for (int p = 0; p < P->npairs; ++p) {
    int n = g->nphi[P->pair_n[p]];
    auto it = lens.find(n);
    if (it == lens.end()) it = lens.emplace(n, (int)lens.size()).first;
    pf[p] = it->second;
  }
  P->nfft = (int)lens.size();
  // kernel limits and radix constants first: the spectra below already run the FFT
  CUDA_TRY(fft_prepare_device(P->device));
  std::vector<FftPlanDev> fps(P->nfft);
  FftPlanDev *scratch = nullptr;
  CUDA_TRY(cudaMalloc(&scratch, sizeof(FftPlanDev)));
  P->fft_allocs.push_back(scratch);
  int maxlen = 0;
  for (auto &kv : lens) {
    if ((rc = build_fft_plan(P, kv.first, fps[kv.second], scratch)) != SHT_OK) return rc;
    maxlen = std::max(maxlen, fps[kv.second].len);
  }
  if ((rc = upload(P, fps, &P->d_fft)) != SHT_OK) return rc;
  if ((rc = upload(P, pf, &P->d_pair_fft)) != SHT_OK) return rc;
  if (maxlen <= kFftMaxLen) {
    P->fft_smem = maxlen * (int)sizeof(double2);
  } else {  // rings beyond shared memory: one L2-resident scratch slot per SM (one CTA each)
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device));
    P->fft_slots = sms;
    P->fft_slot_len = maxlen;
    const size_t bytes = (size_t)sms * maxlen * sizeof(double2);
    CUDA_TRY(cudaMalloc(&P->d_fft_scratch, bytes));
    P->workspace += bytes;
  }
  P->pair_len.resize(P->npairs);
  for (int p = 0; p < P->npairs; ++p) {
    int n = g->nphi[P->pair_n[p]];
    if (P->pair_s[p] >= 0) n = std::max(n, g->nphi[P->pair_s[p]]);
    P->pair_len[p] = n;
  }
  return SHT_OK;
}

extern "C" int sht_plan_create(sht_geom_t geom, sht_alm_t alm, int spin, int ncomp, int precision,
                               sht_plan_t *out) {
  if (!out) return fail(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!geom || !alm) return fail(SHT_ERR_INVALID_ARG, "geometry or a_lm descriptor is NULL");
  if (precision != SHT_FP64 && precision != SHT_MIXED) return fail(SHT_ERR_INVALID_ARG, "bad precision");
  if (ncomp < 1 || ncomp > kMaxJobs) return fail(SHT_ERR_INVALID_ARG, "ncomp must be in 1..%d", kMaxJobs);
  if (abs(spin) > alm->lmax) return fail(SHT_ERR_UNSUPPORTED, "|spin| > lmax");
  if (abs(spin) > 64) return fail(SHT_ERR_UNSUPPORTED, "|spin| > 64");
  if (spin != 0 && ncomp > 8) return fail(SHT_ERR_UNSUPPORTED, "spin transforms take at most 8 (E,B) pairs");
  auto *P = new sht_plan_s;
  cudaGetDevice(&P->device);
  if (cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess || P->sms < 1)
    P->sms = 1;
  P->lmax = alm->lmax;
  P->mmax = alm->mmax;
  P->nm = alm->nm;
  P->astride = alm->stride;
  P->mval = alm->mval;
  P->mstart = alm->mstart;
  P->spin = spin;
  P->ncomp = ncomp;
  P->precision = precision;
  P->fft_df = precision == SHT_MIXED;
  P->nmaps = spin ? 2 * ncomp : ncomp;
  P->njobs_pad = 1;
  while (P->njobs_pad < ncomp) P->njobs_pad *= 2;
  P->nmaps_pad = spin ? 2 * P->njobs_pad : P->njobs_pad;
  int rc = plan_build(P, geom);
  if (rc != SHT_OK) {
    cudaGetLastError();
    free_plan(P);
    return rc;
  }
  *out = P;
  return SHT_OK;
}

// ---- analysis tiling -------------------------------------------------------
static int retile(sht_plan_s *P, int ppt) {
  if (P->batch_refs)
    return fail(SHT_ERR_INVALID_ARG, "the plan belongs to %d batch(es); destroy them before changing its tiling",
                P->batch_refs);
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) CUDA_TRY(cudaSetDevice(P->device));
  const int rc = build_ana_lists(P, ppt);
  if (cur != P->device) cudaSetDevice(cur);
  return rc;
}

extern "C" int sht_plan_set_tiling(sht_plan_t P, int pairs_per_thread) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  const auto c = ana_ppt_candidates(P->spin, P->njobs_pad);
  if (std::find(c.begin(), c.end(), pairs_per_thread) == c.end())
    return fail(SHT_ERR_UNSUPPORTED, "no analysis kernel with %d ring pairs per thread for this plan",
                pairs_per_thread);
  if (pairs_per_thread == P->ana_ppt) return SHT_OK;
  if (P->tc_ana)
    return fail(SHT_ERR_UNSUPPORTED, "the tensor-core analysis takes one ring pair per thread");
  return retile(P, pairs_per_thread);
}

extern "C" int sht_plan_get_tiling(sht_plan_t P, int *pairs_per_thread, int *ncandidates, int *candidates) {
  if (!P || !pairs_per_thread) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *pairs_per_thread = P->ana_ppt;
  const auto c = ana_ppt_candidates(P->spin, P->njobs_pad);
  if (ncandidates) *ncandidates = (int)c.size();
  if (candidates)
    for (size_t i = 0; i < c.size(); ++i) candidates[i] = c[i];
  return SHT_OK;
}

extern "C" int sht_plan_set_fp64_columns(sht_plan_t P, int m_below) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (P->precision != SHT_MIXED) return fail(SHT_ERR_INVALID_ARG, "only mixed-form plans have FP64 columns");
  if (m_below < 0) return fail(SHT_ERR_INVALID_ARG, "m_below must be >= 0");
  if (P->batch_refs)
    return fail(SHT_ERR_INVALID_ARG, "the plan belongs to %d batch(es); destroy them first", P->batch_refs);
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) CUDA_TRY(cudaSetDevice(P->device));
  int rc = SHT_OK;
  // the FP64 tables (coefficients; at spin s the P = E+iB, M = E-iB table the FP64
  // spin kernels read) must reach the new columns: regrow them to the new prefix
  const int64_t need = fp64_prefix(P, m_below);
  if (need > P->ncoef64 || (P->spin != 0 && !P->d_pm64 && m_below > 0)) {
    const int64_t n = std::max(need, P->ncoef64);
    Coef *coef = nullptr;
    double2 *pm = nullptr;
    if (cudaMalloc(&coef, std::max<int64_t>(1, n) * sizeof(Coef)) != cudaSuccess) {
      rc = fail(SHT_ERR_OOM, "FP64 coefficient table");
    } else if (P->spin != 0 &&
               cudaMalloc(&pm, std::max<int64_t>(1, n) * P->nmaps_pad * sizeof(double2)) != cudaSuccess) {
      cudaFree(coef);
      rc = fail(SHT_ERR_OOM, "P/M table");
    } else {
      cudaFree(P->d_coef);
      P->workspace += (n - P->ncoef64) * (int64_t)sizeof(Coef);
      P->d_coef = coef;
      if (P->spin != 0) {
        if (P->d_pm64) {
          cudaFree(P->d_pm64);
          P->workspace -= P->ncoef64 * P->nmaps_pad * (int64_t)sizeof(double2);
        }
        P->d_pm64 = pm;
        P->workspace += n * P->nmaps_pad * (int64_t)sizeof(double2);
      }
      P->ncoef64 = n;
      cudaError_t e = launch_coef_tables(P, 0);  // the FP64 coefficients of the new prefix
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      if (e != cudaSuccess) rc = fail(SHT_ERR_CUDA, "coefficient tables: %s", cudaGetErrorString(e));
    }
  }
  if (rc == SHT_OK) {
    P->fp64_m_below = m_below;
    rc = build_syn_lists(P);
    if (rc == SHT_OK) rc = build_ana_lists(P, P->ana_ppt);
  }
  if (cur != P->device) cudaSetDevice(cur);
  return rc;
}

extern "C" int sht_plan_get_fp64_columns(sht_plan_t P, int *m_below) {
  if (!P || !m_below) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *m_below = P->fp64_m_below;
  return SHT_OK;
}

extern "C" int sht_plan_set_fft_precision(sht_plan_t P, int precision) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (precision != SHT_FP64 && precision != SHT_MIXED) return fail(SHT_ERR_INVALID_ARG, "bad FFT precision");
  if (precision == SHT_MIXED && P->precision != SHT_MIXED)
    return fail(SHT_ERR_INVALID_ARG, "FP64 plans have no double-float FFT tables");
  if (P->batch_refs)
    return fail(SHT_ERR_INVALID_ARG, "the plan belongs to %d batch(es); destroy them first", P->batch_refs);
  P->fft_df = precision == SHT_MIXED;
  return SHT_OK;
}

extern "C" int sht_plan_get_fft_precision(sht_plan_t P, int *precision) {
  if (!P || !precision) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *precision = P->fft_df ? SHT_MIXED : SHT_FP64;
  return SHT_OK;
}

extern "C" int sht_plan_set_tensor_cores(sht_plan_t P, int on) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (on && P->precision != SHT_MIXED) return fail(SHT_ERR_INVALID_ARG, "FP64 plans have no tensor-core form");
  if (on && !tc_supported(P->spin, P->njobs_pad))
    return fail(SHT_ERR_UNSUPPORTED, "tensor-core synthesis holds at most 32 columns (spin 0: ncomp <= 8, spin: ncomp <= 4)");
  if (P->batch_refs)
    return fail(SHT_ERR_INVALID_ARG, "the plan belongs to %d batch(es); destroy them first", P->batch_refs);
  P->tc_syn = on ? 1 : 0;
  return SHT_OK;
}

extern "C" int sht_plan_set_tensor_core_analysis(sht_plan_t P, int on) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (on && P->precision != SHT_MIXED) return fail(SHT_ERR_INVALID_ARG, "FP64 plans have no tensor-core form");
  if (on && !tc_ana_supported(P->spin, P->njobs_pad))
    return fail(SHT_ERR_UNSUPPORTED, "tensor-core analysis holds at most two jobs (ncomp <= 2)");
  if (P->batch_refs)
    return fail(SHT_ERR_INVALID_ARG, "the plan belongs to %d batch(es); destroy them first", P->batch_refs);
  if (on && P->ana_ppt != 1) {  // its tiles: one ring pair per thread
    const int rc = retile(P, 1);
    if (rc != SHT_OK) return rc;
  }
  P->tc_ana = on ? 1 : 0;
  return SHT_OK;
}

extern "C" int sht_plan_get_tensor_core_analysis(sht_plan_t P, int *on) {
  if (!P || !on) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *on = P->tc_ana;
  return SHT_OK;
}

extern "C" int sht_plan_get_tensor_cores(sht_plan_t P, int *on) {
  if (!P || !on) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *on = P->tc_syn;
  return SHT_OK;
}

extern "C" int sht_plan_device_status(sht_plan_t P, int *status) {
  if (!P || !status) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) CUDA_TRY(cudaSetDevice(P->device));
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, P->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(P->d_err, 0, sizeof(int));
  if (cur != P->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return fail(SHT_ERR_CUDA, "device status: %s", cudaGetErrorString(e));
  *status = v;
  return v ? fail(SHT_ERR_TIMEOUT, "a bounded device-side wait gave up (status %d)", v) : SHT_OK;
}

extern "C" int sht_plan_autotune(sht_plan_t P, void *stream, float *ms_per_candidate) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (P->batch_refs) return retile(P, P->ana_ppt);  // reports the error
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) CUDA_TRY(cudaSetDevice(P->device));
  cudaStream_t st = (cudaStream_t)stream;
  const auto cands = ana_ppt_candidates(P->spin, P->njobs_pad);
  // the analysis kernels read the phase array: give it defined contents
  const size_t nph = (size_t)P->nmaps_pad * P->nm * P->npairs * 2;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int rc = SHT_OK, best = P->ana_ppt;
  float best_ms = 0.f;
  cudaError_t e = cudaMemsetAsync(P->d_phase, 0, std::max<size_t>(1, nph) * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  DevPtrs none;
  memset(&none, 0, sizeof(none));
  // the tiling candidates with the double-float analysis, then (mixed plans of
  // supported shapes) the tensor-core analysis on tiles of one pair per thread
  const bool tc_cand = P->precision == SHT_MIXED && tc_ana_supported(P->spin, P->njobs_pad);
  const size_t ncand = cands.size() + (tc_cand ? 1 : 0);
  int best_tc = P->tc_ana;
  if (ms_per_candidate)
    for (size_t i = 0; i <= cands.size(); ++i) ms_per_candidate[i] = 0.f;
  for (size_t i = 0; i < ncand && e == cudaSuccess && rc == SHT_OK; ++i) {
    const bool tc = i == cands.size();
    const int ppt = tc ? 1 : cands[i];
    P->tc_ana = tc ? 1 : 0;
    if ((rc = build_ana_lists(P, ppt)) != SHT_OK) break;
    // one untimed and two timed runs of the analysis Legendre stage (polar cut on)
    for (int it = 0; it < 3 && e == cudaSuccess; ++it) {
      if (it == 1) e = cudaEventRecord(ev[0], st);
      // the tiling's own kernel only (a mixed plan's FP64 items run beside it)
      if (e == cudaSuccess)
        e = P->precision == SHT_MIXED ? launch_leg_ana_mixed(P, none, 1, st) : launch_leg_ana_fp64(P, none, 1, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (ms_per_candidate) ms_per_candidate[i] = ms / 2;
    if (e == cudaSuccess && (i == 0 || ms < best_ms)) {
      best_ms = ms;
      best = ppt;
      best_tc = tc ? 1 : 0;
    }
  }
  P->tc_ana = best_tc;
  if (rc == SHT_OK && e == cudaSuccess && P->ana_ppt != best) rc = build_ana_lists(P, best);
  for (auto x : ev)
    if (x) cudaEventDestroy(x);
  if (cur != P->device) cudaSetDevice(cur);
  if (rc != SHT_OK) return rc;
  if (e != cudaSuccess) return fail(SHT_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  return SHT_OK;
}

extern "C" int sht_plan_workspace(sht_plan_t P, int64_t *bytes) {
  if (!P || !bytes) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *bytes = P->workspace;
  return SHT_OK;
}

extern "C" int sht_plan_triples(sht_plan_t P, int flags, int64_t *t) {
  if (!P || !t) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *t = P->triples[(flags & SHT_NO_POLAR_OPT) ? 0 : 1];
  return SHT_OK;
}

extern "C" int sht_plan_triples_joined(sht_plan_t P, int64_t *t) {
  if (!P || !t) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  *t = P->precision == SHT_MIXED ? P->triples_joined : P->triples[1];
  return SHT_OK;
}

extern "C" void sht_plan_destroy(sht_plan_t P) { free_plan(P); }

extern "C" int sht_plan_profile(sht_plan_t P, int enable) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  for (auto &r : P->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  P->prof.clear();
  P->prof_on = enable ? 1 : 0;
  return SHT_OK;
}

extern "C" int sht_plan_profile_read(sht_plan_t P, double *ms, int64_t *count) {
  if (!P || !ms || !count) return fail(SHT_ERR_INVALID_ARG, "NULL argument");
  for (int s = 0; s < SHT_NSTAGES; ++s) {
    ms[s] = 0.0;
    count[s] = 0;
  }
  int rc = SHT_OK;
  for (auto &r : P->prof) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && rc == SHT_OK) rc = fail(SHT_ERR_CUDA, "profile events: %s", cudaGetErrorString(e));
    ms[r.stage] += t;
    count[r.stage] += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  P->prof.clear();
  return rc;
}

// ----------------------------------------------------------------------------
// Execution
// ----------------------------------------------------------------------------
extern "C" int sht_execute(sht_plan_t P, int type, double *const *alm, double *const *map, int flags,
                           void *stream) {
  if (!P) return fail(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (type < SHT_SYNTHESIS || type > SHT_DERIV_SYNTHESIS) return fail(SHT_ERR_INVALID_ARG, "bad type %d", type);
  const bool deriv = type == SHT_DERIV_SYNTHESIS;
  if (deriv && P->spin != 1) return fail(SHT_ERR_INVALID_ARG, "SHT_DERIV_SYNTHESIS needs a plan of spin 1");
  if (flags & ~(SHT_ADD_OUTPUT | SHT_NO_POLAR_OPT | SHT_REAL_HARMONICS | SHT_GRADIENT))
    return fail(SHT_ERR_INVALID_ARG, "unknown flags");
  const bool real = (flags & SHT_REAL_HARMONICS) != 0;
  const bool grad = (flags & SHT_GRADIENT) != 0;
  if (grad && ((type != SHT_ADJOINT_SYNTHESIS && type != SHT_ADJOINT_ANALYSIS) || real))
    return fail(SHT_ERR_INVALID_ARG, "SHT_GRADIENT applies to the two adjoint types in complex storage only");
  if (!alm || !map) return fail(SHT_ERR_INVALID_ARG, "pointer arrays are NULL");
  DevPtrs A, M;
  memset(&A, 0, sizeof(A));
  memset(&M, 0, sizeof(M));
  const int nin = deriv ? P->ncomp : P->nmaps;  // a_lm arrays read
  for (int j = 0; j < P->nmaps; ++j) {
    if (!map[j] || (j < nin && !alm[j])) return fail(SHT_ERR_INVALID_ARG, "NULL device pointer at index %d", j);
    if (j < nin) A.p[j] = alm[j];
    M.p[j] = map[j];
  }
  // padding jobs (kernels run a power-of-two job count) read job 0's input;
  // their results stay in the plan's workspace and are never written out
  const int per = (P->spin && !deriv) ? 2 : 1;
  for (int j = nin; j < P->nmaps_pad; ++j) A.p[j] = alm[j % per];
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) CUDA_TRY(cudaSetDevice(P->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int polar = (flags & SHT_NO_POLAR_OPT) ? 0 : 1;
  const int add = (flags & SHT_ADD_OUTPUT) ? 1 : 0;
  cudaError_t e = cudaSuccess;
  // run one stage on stream s, bracketed by an event pair on s when profiling
  auto stage = [&](int id, cudaStream_t s, auto &&launch) {
    if (e != cudaSuccess) return;
    sht_plan_s::ProfRec r{id, nullptr, nullptr};
    if (P->prof_on) {
      if ((e = cudaEventCreate(&r.a)) != cudaSuccess) return;
      if ((e = cudaEventCreate(&r.b)) != cudaSuccess) return;
      if ((e = cudaEventRecord(r.a, s)) != cudaSuccess) return;
    }
    e = launch();
    if (P->prof_on) {
      if (e == cudaSuccess) e = cudaEventRecord(r.b, s);
      P->prof.push_back(r);
    }
  };
  auto record = [&](cudaEvent_t ev, cudaStream_t s) {
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
  };
  auto wait = [&](cudaStream_t s, cudaEvent_t ev) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
  };
  const bool mixed = P->precision == SHT_MIXED;
  // a_lm read by a synthesis: derivative mode, real storage, or (the adjoint
  // analysis of a gradient) the m > 0 entries halved
  const int mode = (deriv ? kAlmDeriv : 0) | (real ? kAlmReal : 0) | (grad ? kAlmHalf : 0);
  const int amode = mode & (kAlmReal | kAlmHalf);
  auto leg = [&](int stg, const void *items, int n, cudaStream_t s) {
    return mixed ? launch_leg_mixed_items(P, stg, polar, items, n, s)
                 : launch_leg_fp64_items(P, stg, A, polar, items, n, s, amode);
  };
  // A mixed plan's FP64 items (small m near the poles) run on the high-priority
  // side stream beside its mixed Legendre kernel; the ring FFT waits for both.
  if (type == SHT_SYNTHESIS || type == SHT_ADJOINT_ANALYSIS || deriv) {
    const int weighted = type == SHT_ADJOINT_ANALYSIS;
    const bool lo = mixed && P->nsyn_lo[polar] > 0;
    stage(0, st, [&] {
      cudaError_t r = mixed ? launch_alm_prepare_mixed(P, A, st, mode) : launch_alm_prepare_fp64(P, A, st, mode);
      if (r == cudaSuccess && lo) r = launch_alm_prepare_fp64(P, A, st, mode);  // the FP64 items read P/M
      return r;
    });
    if (lo) {
      record(P->ev_fork, st);
      wait(P->side, P->ev_fork);
      stage(5, P->side, [&] {
        return launch_leg_fp64_items(P, 0, A, polar, P->d_syn_lo[polar], P->nsyn_lo[polar], P->side, amode);
      });
      record(P->ev_lo, P->side);
    }
    stage(0, st, [&] { return leg(0, P->d_syn_items[polar], P->nsyn_items[polar], st); });
    if (lo) wait(st, P->ev_lo);
    stage(1, st, [&] { return launch_fft_syn(P, M, polar, weighted, add, st); });
  } else {
    const int weighted = type == SHT_ANALYSIS;
    const bool lo = mixed && P->nana_lo[polar] > 0;
    stage(2, st, [&] { return launch_fft_ana(P, M, weighted, st); });
    if (lo) {
      record(P->ev_fork, st);
      wait(P->side, P->ev_fork);
      stage(5, P->side, [&] {
        return launch_leg_fp64_items(P, 1, A, polar, P->d_ana_lo[polar], P->nana_lo[polar], P->side);
      });
      record(P->ev_lo, P->side);
    }
    stage(3, st, [&] { return leg(1, P->d_ana_items[polar], P->nana_items[polar], st); });
    if (lo) wait(st, P->ev_lo);
    stage(4, st, [&] { return launch_ana_reduce(P, A, polar, add, st, real, grad); });
  }
  if (cur != P->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return fail(SHT_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return SHT_OK;
}
