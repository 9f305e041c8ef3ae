/*
 * sht_gb300.h -- C ABI of the GB300 (sm_103a) spherical harmonic transform library.
 *
 * The problem statement follows Reinecke & Seljebotn 2013, "Libsharp --
 * spherical harmonic transforms revisited", Sect. 2:
 *
 *   synthesis (Eq. syn_used)
 *     p_xy = sum_{m=-lmax}^{lmax} sum_{l>=|m|} sa_lm  sLambda_lm(theta_y)
 *            exp(i m phi0_y + 2 pi i m x / Nphi_y)
 *   analysis (Eq. ana_used)
 *     sa_lm = sum_y sum_x p_xy w_y sLambda_lm(theta_y) exp(-i m phi0_y - 2 pi i m x / Nphi_y)
 *
 * with sLambda_lm(theta) = sY_lm(theta, 0) = (-1)^m sqrt((2l+1)/(4 pi)) d^l_{-m,s}(theta)
 * (Sect. 4.1), on any iso-latitude grid (Sect. 2 and 4.4): ring y has
 * colatitude theta_y, Nphi_y equidistant pixels starting at azimuth phi0_y,
 * a quadrature weight w_y, and its pixels live at map[ofs_y + x * stride_y].
 *
 * Conventions (no C99 complex type appears in this interface, Sect. 3.1):
 *  - a_lm are complex numbers stored as interleaved (re, im) doubles, only for
 *    m >= 0; for a listed m the coefficient a_lm sits at complex index
 *    mstart[m_index] + l * stride (l = m..lmax).  The default layout is the
 *    triangular m-major one, index m (2 lmax + 1 - m) / 2 + l.
 *  - Maps are real doubles.  The imaginary part of a_l0 is ignored on input
 *    and written as 0 on output (real fields).
 *  - spin s != 0: ncomp counts (E, B) pairs.  alm[2k], alm[2k+1] are E and B,
 *    map[2k], map[2k+1] are Q and U, with
 *        sa = -(E + iB),  (-s)a = -(-1)^s (E - iB),  Q + iU = sum sa_lm sY_lm.
 *    spin 0: alm[k] and map[k], k < ncomp.
 *  - All a_lm and map pointers passed to sht_execute are DEVICE pointers on
 *    the device that was current when the plan was made; the arrays of
 *    pointers themselves are host memory.  The caller owns these buffers.
 *  - Geometry, a_lm descriptor and plan handles are owned by the library
 *    until the matching *_destroy call.  A plan copies what it needs from the
 *    geometry and a_lm descriptors, which may be destroyed right after.
 *  - Every function returns SHT_OK (0) or a negative error code; no
 *    exceptions cross this boundary.  sht_strerror() names the code and
 *    sht_last_error() gives a message for the last failure on this thread.
 *
 * This header is shared by the C/C++ caller and the Python binding; it names
 * no CUDA or torch type (streams are passed as void*).
 */
#ifndef SHT_GB300_H
#define SHT_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define SHT_API __attribute__((visibility("default")))
#else
#define SHT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SHT_OK 0
#define SHT_ERR_INVALID_ARG -1  /* a size, index, pointer or enum is out of range */
#define SHT_ERR_UNSUPPORTED -2  /* valid request the library does not implement (e.g. spin > lmax, an FFT length it cannot factor) */
#define SHT_ERR_OOM -3          /* device or host allocation failed */
#define SHT_ERR_CUDA -4         /* a CUDA runtime call or kernel launch failed */
#define SHT_ERR_TIMEOUT -5      /* a bounded device-side wait gave up */

/* ---- enums ------------------------------------------------------------- */
#define SHT_ECP_FEJER1 0 /* theta_n = (n + 1/2) pi / nlat, n = 0..nlat-1 (Sect. 4.4.1) */
#define SHT_ECP_FEJER2 1 /* theta_n = n pi / (nlat + 1),  n = 1..nlat */
#define SHT_ECP_CC 2     /* theta_n = n pi / (nlat - 1),  n = 0..nlat-1 (Clenshaw-Curtis) */

#define SHT_FP64 0  /* recursion and accumulation in IEEE double */
#define SHT_MIXED 1 /* recursion, accumulation and (by default) ring FFTs in compensated FP32 pairs; FP64 kept for tables and start values */

#define SHT_SYNTHESIS 0         /* a_lm -> map, Eq. syn_used */
#define SHT_ANALYSIS 1          /* map -> a_lm, Eq. ana_used (with the ring weights) */
#define SHT_ADJOINT_SYNTHESIS 2 /* map -> a_lm, Y^T p: analysis with all weights 1 (Sect. 4.5) */
#define SHT_ADJOINT_ANALYSIS 3  /* a_lm -> map, W Y a: synthesis times the ring weights (Sect. 4.5) */
/* spin-0 a_lm -> the two maps df/dtheta and df/(sin(theta) dphi) (Sect. 4.3); plans of spin 1:
 * the spin-1 synthesis of E = sqrt(l(l+1)) a_lm, B = 0 (with the E/B convention of reading R5,
 * Q + iU = -sum E_lm 1Y_lm = (d/dtheta + i/sin(theta) d/dphi) f).  alm[] holds ncomp arrays,
 * map[] 2 ncomp (derivative in theta, then in phi, per component). */
#define SHT_DERIV_SYNTHESIS 4

#define SHT_ADD_OUTPUT 1   /* add the result to the output arrays instead of overwriting them */
#define SHT_NO_POLAR_OPT 2 /* evaluate every (m, ring) term, skipping none (Sect. 3.3) */
/* a_lm in real-harmonic storage (Sect. 4.5; the paper defers the definition, this
 * is the reading taken): for m > 0 the two doubles of a coefficient hold
 * [a_{l,m}, a_{l,-m}] = sqrt(2) (Re a_lm, -Im a_lm), the coefficients of the
 * orthonormal real basis sqrt(2) Re Y_lm, sqrt(2) Im Y_lm; m = 0 entries are
 * unchanged.  Inputs are read and outputs written in that storage; with it the
 * adjoint synthesis is the exact transpose of the synthesis under the plain dot
 * product of the stored numbers.  sht_execute and sht_execute_noalloc only. */
#define SHT_REAL_HARMONICS 4
/* The gradient factors of the adjoint transforms (Sect. 4.5), for a real loss L
 * of real maps with the a_lm stored for m >= 0 only: the synthesis counts every
 * stored m > 0 coefficient twice (once for -m), so with D = diag(2 - delta_m0)
 *   SHT_ADJOINT_SYNTHESIS | SHT_GRADIENT writes D Y^H g = dL/da for g = dL/dp
 *     (dL/da = dL/dRe a + i dL/dIm a; the m = 0 entries' imaginary part is 0),
 *   SHT_ADJOINT_ANALYSIS | SHT_GRADIENT reads g = dL/da of an analysis a = A p
 *     and writes W S D^-1 g = dL/dp (the m > 0 entries count half).
 * Only these two types and complex storage (not with SHT_REAL_HARMONICS, whose
 * adjoint already is the gradient); sht_execute only. */
#define SHT_GRADIENT 8

typedef struct sht_geom_s *sht_geom_t;
typedef struct sht_alm_s *sht_alm_t;
typedef struct sht_plan_s *sht_plan_t;
typedef struct sht_batch_s *sht_batch_t;

/* ---- geometry (Sect. 2, Sect. 4.4) -------------------------------------- */

/*
 * General iso-latitude grid; partial coverage is allowed (any subset of rings).
 * theta[nrings] in (0, pi) or [0, pi]; nphi[nrings] >= 1; phi0[nrings] radians;
 * ofs[nrings] index of pixel 0 of the ring in each map; stride[nrings] pixel
 * stride (may be NULL: all 1); weight[nrings] quadrature weight per pixel
 * (may be NULL: all 1; the user is responsible for correct weights, Sect. 4.4).
 * Rings whose colatitudes mirror each other (theta' = pi - theta within 1e-12
 * rad) and have equal nphi are processed as north/south pairs.
 * Host arrays, copied.  Errors: SHT_ERR_INVALID_ARG.
 */
SHT_API int sht_geom_general(int nrings, const double *theta, const int *nphi, const double *phi0,
                     const int64_t *ofs, const int *stride, const double *weight, sht_geom_t *out);

/*
 * Gauss-Legendre grid (Sect. 4.4, used throughout Sect. 5): nlat rings at the
 * roots of P_nlat, north to south, nlon pixels each, phi0 = 0, contiguous
 * ring-major map (ofs = y * nlon), weight = Gauss weight * 2 pi / nlon.
 */
SHT_API int sht_geom_gauss(int nlat, int nlon, sht_geom_t *out);

/*
 * Reduced Gauss-Legendre grid (Sect. 4.4.2): the nlat Gauss-Legendre rings of
 * sht_geom_gauss, each thinned to the smallest 2^a 3^b 5^c >= 2 m_y + 1
 * pixels, where m_y = min(lmax, s cos(theta) + sqrt((T + lmax sin(theta))^2 -
 * s^2 sin^2(theta))) solves Eq. eq_polaropt for m (T = max(100, 0.01 lmax), s =
 * |spin|); weight w_GL 2 pi / Nphi_y, phi0 = 0, rings stored one after another.
 * Not exact in the mathematical sense, exact to the precision the polar
 * optimisation keeps.  Errors: SHT_ERR_INVALID_ARG, SHT_ERR_OOM.
 */
SHT_API int sht_geom_reduced_gauss(int nlat, int lmax, int spin, sht_geom_t *out);

/*
 * ECP grid (Sect. 4.4.1): kind SHT_ECP_FEJER1 / FEJER2 / CC, nlat rings,
 * nlon pixels each, phi0 = 0, contiguous ring-major map, weights of
 * Fejer's first / second rule or Clenshaw-Curtis times 2 pi / nlon.
 */
SHT_API int sht_geom_ecp(int kind, int nlat, int nlon, sht_geom_t *out);

/*
 * HEALPix grid (named in Sect. 1 and 4.4; ring layout of Gorski et al. 2005):
 * 4 nside - 1 rings, RING pixel order, polar rings Nphi = 4i with
 * phi0 = pi/(4i), equatorial rings Nphi = 4 nside with phi0 = pi/(4 nside) for
 * even (i - nside) and 0 for odd, weight 4 pi / (12 nside^2) per pixel.
 */
SHT_API int sht_geom_healpix(int nside, sht_geom_t *out);

/* Partial coverage: a new geometry holding rings[0..nsel-1] of g (pixel offsets kept). */
SHT_API int sht_geom_subset(sht_geom_t g, int nsel, const int *rings, sht_geom_t *out);

/* Ring count, total pixel span (max over rings of ofs + (nphi-1)*stride + 1) and number of ring pairs. */
SHT_API int sht_geom_info(sht_geom_t g, int *nrings, int64_t *npix, int *npairs);

/* Copy out the per-ring description (any pointer may be NULL). */
SHT_API int sht_geom_rings(sht_geom_t g, double *theta, int *nphi, double *phi0, int64_t *ofs,
                   int *stride, double *weight);

SHT_API void sht_geom_destroy(sht_geom_t g);

/* ---- a_lm layout (any subset of m may be listed, e.g. a round-robin share, Sect. 4.2) */

/*
 * lmax >= 0, 0 <= mmax <= lmax.  nm = number of listed m (mval == NULL: all
 * m = 0..mmax, nm ignored).  mval[nm] distinct values in [0, mmax];
 * mstart[nm] (NULL: triangular layout over the listed m, see above);
 * stride = complex stride in l (>= 1).
 */
SHT_API int sht_alm_create(int lmax, int mmax, int nm, const int *mval, const int64_t *mstart, int stride,
                   sht_alm_t *out);

/* Number of complex entries an array must hold for this layout. */
SHT_API int sht_alm_size(sht_alm_t a, int64_t *ncomplex);

SHT_API void sht_alm_destroy(sht_alm_t a);

/* ---- plan and execution -------------------------------------------------- */

/*
 * Plan a transform on the current CUDA device: spin s (|s| <= lmax,
 * |s| <= 64), ncomp simultaneous transforms of identical type (1..16; Sect. 3.2),
 * precision SHT_FP64 or SHT_MIXED.  Builds, on the device, the recursion
 * coefficient tables for every listed m and l (Sect. 4.1), the ring-pair
 * list, the polar-optimisation ranges (Sect. 3.3) and the ring FFT plans.
 * Errors: SHT_ERR_INVALID_ARG, SHT_ERR_UNSUPPORTED (e.g. a ring length the FFT
 * cannot handle), SHT_ERR_OOM, SHT_ERR_CUDA.
 */
SHT_API int sht_plan_create(sht_geom_t geom, sht_alm_t alm, int spin, int ncomp, int precision,
                    sht_plan_t *out);

/*
 * Run one transform of the planned kind on stream cuda_stream (a cudaStream_t,
 * NULL = legacy default stream).  type is one of SHT_SYNTHESIS, SHT_ANALYSIS,
 * SHT_ADJOINT_SYNTHESIS, SHT_ADJOINT_ANALYSIS, or SHT_DERIV_SYNTHESIS (spin-1
 * plans only: ncomp spin-0 a_lm arrays in, 2 ncomp maps out); alm[] / map[]
 * hold ncomp (spin 0) or 2 ncomp (spin != 0) device pointers.  Inputs are read, outputs
 * overwritten (or accumulated with SHT_ADD_OUTPUT); pixels and a_lm entries
 * outside the geometry / layout are not touched.  Asynchronous: returns after
 * the launches are queued.  Calls that share a plan must not overlap (they use
 * the plan's workspace).  Errors: SHT_ERR_INVALID_ARG, SHT_ERR_CUDA.
 */
SHT_API int sht_execute(sht_plan_t plan, int type, double *const *alm, double *const *map, int flags,
                void *cuda_stream);

/* Bytes of device workspace the plan holds: coefficient tables, the phase array,
 * the analysis partial sums and, for a mixed plan, the recursion state where each
 * (m, ring pair)'s terms start (48 bytes each, built once at plan creation so the
 * Legendre kernels skip the negligible stretch of the recursion). */
SHT_API int sht_plan_workspace(sht_plan_t plan, int64_t *bytes);

/*
 * Exact algorithmic work of one transform of this plan: the number of
 * (m, l, ring-pair) recursion steps after the polar cut (flags as for
 * sht_execute; SHT_NO_POLAR_OPT counts every step).
 */
SHT_API int sht_plan_triples(sht_plan_t plan, int flags, int64_t *triples);

/*
 * The part of that work a mixed plan's Legendre kernels cannot skip: the steps
 * from each kept pair's join block on (the first block of 16 degrees from l0 with
 * terms that are not negligible; before it a pair adds nothing), the polar cut
 * applied.  The kernels walk a CTA (or a warp) from its pairs' earliest join block,
 * so they run somewhat more steps than this.  An FP64 plan reports its
 * sht_plan_triples count.  Errors: SHT_ERR_INVALID_ARG.
 */
SHT_API int sht_plan_triples_joined(sht_plan_t plan, int64_t *triples);

SHT_API void sht_plan_destroy(sht_plan_t plan);

/* ---- analysis tiling and autotuning -------------------------------------------
 * The paper tunes its kernels by hand for each CPU; here the one shape the
 * analysis Legendre kernel leaves open -- how many ring pairs each thread
 * walks (more pairs amortise the per-degree reduction across the CTA, fewer
 * leave room for more resident warps) -- is chosen per plan by measurement.
 * A plan offers the tilings its kernels are built for (1 to 3 values,
 * depending on spin class and ncomp); the first is the default.
 *
 * sht_plan_get_tiling writes the current pairs per thread and, when the
 * pointers are not NULL, the number of candidates and the candidates (at most
 * 4).  sht_plan_set_tiling selects a candidate (SHT_ERR_UNSUPPORTED for any
 * other value, and for any value but 1 while the tensor-core analysis is on).
 * sht_plan_autotune runs the plan's analysis Legendre kernel once untimed and
 * twice timed per candidate on cuda_stream -- the tilings with the double-float
 * analysis and, for a mixed plan of a shape the tensor-core analysis supports,
 * that analysis (one pair per thread) -- keeps the fastest (setting
 * sht_plan_set_tensor_core_analysis accordingly) and, if ms_per_candidate is not
 * NULL (room for ncandidates + 1 floats), writes each candidate's time per run,
 * the tensor-core analysis' last (0 where it is no candidate).  It overwrites the plan's phase workspace, synchronises the stream
 * and must not be captured.  Results do not depend on the tiling beyond
 * rounding.  Neither call may change a plan that a batch refers to
 * (SHT_ERR_INVALID_ARG).  Errors: SHT_ERR_INVALID_ARG, SHT_ERR_UNSUPPORTED,
 * SHT_ERR_OOM, SHT_ERR_CUDA.
 */
SHT_API int sht_plan_get_tiling(sht_plan_t plan, int *pairs_per_thread, int *ncandidates, int *candidates);
SHT_API int sht_plan_set_tiling(sht_plan_t plan, int pairs_per_thread);
SHT_API int sht_plan_autotune(sht_plan_t plan, void *cuda_stream, float *ms_per_candidate);

/* ---- FP64 columns of the mixed form --------------------------------------------
 * The paper computes in double precision throughout; the mixed form (not in the
 * paper) runs the recursion and sums in pairs of FP32 numbers, ~48 significant
 * bits.  For small m, on rings near the poles, the recursion is non-oscillatory
 * over l < ~1/theta and amplifies its per-step rounding by a power of l, so those
 * values lose accuracy first as lmax grows.  A mixed plan therefore runs the work
 * items of the columns m < m_below that touch a ring within 0.05 rad of a pole in
 * the FP64 kernels (same results as an FP64 plan there), on a high-priority side
 * stream beside the mixed kernels.  The default is lmax / 170 from lmax 2000 on
 * (12 at lmax 2047, 24 at 4095, 48 at 8191), 0 below: every ring's own error
 * stays near or below 5e-11 (spin-2 synthesis against the FP64 form, ring by
 * ring; the rings nearest the poles need the most columns), and the FP64 items
 * stay hidden beside the mixed kernels.  The plan keeps FP64 coefficients (32
 * bytes per (m, l)) and, at spin s, a P = E+iB, M = E-iB table (16 bytes per (m,
 * l) and array) only for the columns below the bound.  sht_plan_set_fp64_columns
 * changes it (any m_below >= 0; it rebuilds the work lists and, for a higher
 * bound, reallocates those tables, which synchronises the device);
 * sht_plan_get_fp64_columns reads it.
 * Errors: SHT_ERR_INVALID_ARG (NULL, an FP64 plan, a plan in a batch,
 * m_below < 0), SHT_ERR_OOM, SHT_ERR_CUDA.
 */
SHT_API int sht_plan_set_fp64_columns(sht_plan_t plan, int m_below);
SHT_API int sht_plan_get_fp64_columns(sht_plan_t plan, int *m_below);

/* Ring FFT arithmetic of a mixed plan (Eqs. syn1, ana2).  By default a mixed plan
 * runs its ring FFTs in the same double-float arithmetic as its Legendre stage
 * (FP32 pairs, ~46 bits an operation: relative errors near 1e-14, far inside the
 * mixed form's 1e-10; values within FP32's normal range, magnitudes below 2^-126
 * entering as zero); on GB300 the FP32 pipe issues 64 times the FP64 rate.
 * sht_plan_set_fft_precision(plan, SHT_FP64) selects the IEEE-double engine the
 * FP64 plans use, SHT_MIXED the double-float one; sht_plan_get_fft_precision
 * reads the setting.  FP64 plans always use the FP64 engine.
 * Errors: SHT_ERR_INVALID_ARG (NULL, an FP64 plan asked for SHT_MIXED, a value
 * other than SHT_FP64 / SHT_MIXED, a plan in a batch).
 */
SHT_API int sht_plan_set_fft_precision(sht_plan_t plan, int precision);
SHT_API int sht_plan_get_fft_precision(sht_plan_t plan, int *precision);

/* ---- the synthesis contraction on the tensor cores ---------------------------
 * The paper's synthesis (Eq. syn2; the inner loop of Sect. 3.2, Fig. 1) is, for
 * one m, a product F = Lambda^T a over the degrees l.  A mixed plan can run that
 * product on the tensor cores: the double-float recursion of Sect. 4.1 still
 * generates Lambda, which is split exactly into three bf16 digits on a grid set
 * by the ring pair's own bound (found once at plan creation) plus an FP32
 * remainder (contracted on the CUDA cores); the a_lm are split into six bf16
 * digits on a grid per 256 degrees; the digit products are summed in FP32
 * accumulators where no rounding can occur, and the sums are added in
 * double-float.  A term's error is below 2^-43 of the bound of its operands; at
 * spin 2, lmax 4095 the maps agree with the FP64 form to 2.1e-12 relative, as
 * with the double-float contraction.
 * Shapes: spin 0 with ncomp <= 8, spin s with ncomp <= 4 (SHT_ERR_UNSUPPORTED
 * otherwise).  It serves SHT_SYNTHESIS, SHT_ADJOINT_ANALYSIS and
 * SHT_DERIV_SYNTHESIS through sht_execute and sht_execute_noalloc, and is a
 * mixed plan's default for every supported shape except a single spin-0 map,
 * where the double-float contraction is faster (measured on GB300 at lmax 4095:
 * spin 2 one E/B pair 54.3 ms against 62.7, spin 0 eight maps 69.9 against 103.7,
 * spin 0 one map 26.3 against 22.2).  sht_plan_set_tensor_cores(plan, 1 or 0)
 * selects it or the double-float contraction; sht_plan_get_tensor_cores reads the
 * setting.  A batch runs each plan with the setting it had when the batch was
 * made (the setting cannot change while a batch refers to the plan).  Errors: SHT_ERR_INVALID_ARG (NULL, an
 * FP64 plan, a plan in a batch), SHT_ERR_UNSUPPORTED.
 *
 * The tensor-core kernel waits on its own matrix products with a bounded number
 * of tries; if a wait gives up it stops, records bit 0 in the plan's device
 * status word and leaves its outputs undefined.  sht_plan_device_status
 * synchronises the device, writes the word to *status, clears it and returns
 * SHT_ERR_TIMEOUT if it was set (SHT_OK otherwise).
 */
SHT_API int sht_plan_set_tensor_cores(sht_plan_t plan, int on);
SHT_API int sht_plan_get_tensor_cores(sht_plan_t plan, int *on);
SHT_API int sht_plan_device_status(sht_plan_t plan, int *status);

/* ---- the analysis contraction on the tensor cores ----------------------------
 * The paper's analysis (Eq. ana1; the loop over rings inside the loop over l,
 * Sect. 3.2, Fig. 2) is, for one m and the ring pairs of a tile, a product
 * a = G Lambda over the ring pairs.  A mixed plan can run it transposed on the
 * tensor cores: the double-float recursion of Sect. 4.1 still generates Lambda,
 * one thread per ring pair, which is split exactly into six bf16 digits of
 * Lambda / u_p (u_p the ring pair's own bound, found once at plan creation);
 * the ring pair's phase values times u_p are split into six bf16 digits on a
 * grid per tile and column; the digit products are summed over the tile's pairs
 * in FP32 accumulators where no rounding can occur, and the levels are added in
 * double-float.  Shapes: ncomp <= 2 (SHT_ERR_UNSUPPORTED otherwise); tiles of
 * one pair per thread (the call sets that tiling).  It serves SHT_ANALYSIS and
 * SHT_ADJOINT_SYNTHESIS through sht_execute, sht_execute_noalloc and the stage
 * call, and in a batch made while the plan has it set.  sht_plan_autotune selects it
 * where it is measured faster (GB300, lmax 4095: spin 2 one E/B pair 73.8 ms
 * against 76.5 for the double-float analysis, two pairs 100.7 against 134.1;
 * spin 0 one map 45.7 against 25.2); sht_plan_set_tensor_core_analysis(plan, 1
 * or 0)
 * sets it, sht_plan_get_tensor_core_analysis reads it.  Its waits are bounded
 * like the synthesis kernel's (status word bit 0).  Errors: SHT_ERR_INVALID_ARG
 * (NULL, an FP64 plan, a plan in a batch), SHT_ERR_UNSUPPORTED, and those of
 * sht_plan_set_tiling.
 */
SHT_API int sht_plan_set_tensor_core_analysis(sht_plan_t plan, int on);
SHT_API int sht_plan_get_tensor_core_analysis(sht_plan_t plan, int *on);

/* ---- measurement ----------------------------------------------------------
 * Sect. 5.2 times whole transforms by wall clock; these two calls report the
 * device time of each kernel stage instead.  While profiling is on,
 * sht_execute records a CUDA event pair around every kernel it launches, on
 * the stream that kernel runs on (stage 0 Legendre synthesis with the a_lm
 * conversion, 1 FFT synthesis, 2 FFT analysis, 3 Legendre analysis, 4 tile
 * reduction of the analysis, 5 the FP64 items of a mixed plan, which overlap
 * stage 0 or 3 on a stream of their own).  enable = 1 starts
 * (and clears) the record, 0 stops it.  sht_plan_profile_read waits for the
 * recorded events, then writes for each stage s < SHT_NSTAGES the summed
 * milliseconds ms[s] and the number of launches count[s], and clears the
 * record.  Errors: SHT_ERR_INVALID_ARG, SHT_ERR_CUDA.
 */
#define SHT_NSTAGES 6
SHT_API int sht_plan_profile(sht_plan_t plan, int enable);
SHT_API int sht_plan_profile_read(sht_plan_t plan, double *ms, int64_t *count);

/* Measured throughput of the pipes the transforms run on (the denominators of
 * their rooflines), on device (-1: the current one): every thread of a grid of 8
 * CTAs x 256 threads per SM runs 8 independent chains of one operation; the
 * best of three timed launches after an untimed one.  out[0] FP64 FMA in
 * TFLOP/s (an FMA counted as 2 flops), out[1] FP32 FMA and out[2] FP32 add in
 * T op/s (one per lane operation, as the mixed form's roofline counts them).
 * Runs on a stream of its own and synchronises it (about 40 ms on a GB300).
 * Errors: SHT_ERR_INVALID_ARG (NULL out, bad device), SHT_ERR_CUDA.
 */
SHT_API int sht_measure_pipe_peaks(int device, double *out);

/* How the ring FFTs (Eqs. syn1, ana2) transform a ring of n points; host logic
 * only, no device needed.  kind: 0 mixed radix of length n, 1 Rader (n prime,
 * n - 1 smooth) of length n - 1, 2 Bluestein (a chirp convolution) of length
 * len >= 2n - 1.  radices[0..nrad) (caller-owned, room for 24) are the passes of
 * the length-len transform in order: 4s, a 2, then odd radices up to 127
 * ascending; their product is len.  Errors: SHT_ERR_INVALID_ARG (NULL, n < 1),
 * SHT_ERR_UNSUPPORTED (no transform of at most 65536 points fits).
 */
SHT_API int sht_fft_plan_info(int n, int *kind, int *len, int *nrad, int *radices);

/* The polar optimisation (Sect. 3.3, Eq. eq_polaropt, T = max(100, 0.01 lmax)) as
 * a plan of this geometry, lmax and spin applies it; host logic only, no device
 * needed.  Ring pairs (sht_geom_info's npairs) are ordered from the poles towards
 * the equator; for each of the nm values mval[i] (0 <= m <= lmax) first_pair[i]
 * is the first pair kept (npairs: none), the cut being a prefix.  pair_theta, if
 * not NULL, receives the northern ring's theta of every pair in that order
 * (npairs doubles).  *triples = sum over m of (npairs - first_pair) (lmax -
 * max(m, |spin|) + 1), the (m, l, ring-pair) steps of one Legendre stage.
 * Arrays are caller-owned.  Errors: SHT_ERR_INVALID_ARG (NULL, lmax < 0, nm < 1,
 * m outside 0..lmax).
 */
SHT_API int sht_geom_polar_cut(sht_geom_t geom, int lmax, int spin, int nm, const int *mval, int *first_pair,
                               double *pair_theta, int64_t *triples);

/* ---- the two stages of a transform (distributed decomposition, Sect. 4.2) --------
 * Sect. 4.2 (Figs. 3 and 4) distributes a transform over tasks: each task runs
 * the Legendre stage for its own m values over all rings, the phase array is
 * rearranged among the tasks so that each holds every m for its own rings, and
 * each task runs the ring FFTs of its rings; an analysis runs the steps
 * backwards.  These two calls are the stages of a plan's transform, with the
 * phase array in caller-owned DEVICE memory in a per-ring layout:
 *   phase[(c * nm + i) * nrings + y]  (complex, interleaved re, im doubles)
 * for map c < nmaps (the maps of sht_execute: ncomp, or 2 ncomp for spin),
 * m = the plan's i-th listed m (sht_alm_create's mval, default 0..mmax), ring y
 * of the plan's geometry.  For a synthesis F holds the ring's Fourier
 * coefficients of Eq. syn2, map_c(y, x) = sum over m = -mmax..mmax of
 * F_{c,m,y} e^{i m (phi0_y + 2 pi x / Nphi_y)} with F_{c,-m} = conj(F_{c,m}) (real
 * maps); for an analysis G_{c,m,y} of Eq. ana2 (ring weights applied for
 * SHT_ANALYSIS, not for SHT_ADJOINT_SYNTHESIS).  A distributed transform uses
 * one plan per task for its m values (a listed-m a_lm layout, the whole
 * geometry) and one for its rings (sht_geom_subset, every m).
 *
 * sht_execute_legendre: SHT_SYNTHESIS / SHT_ADJOINT_ANALYSIS read alm[] and
 * write phase (entries the polar optimisation of Sect. 3.3 skips are written as
 * zero; flags SHT_NO_POLAR_OPT, SHT_REAL_HARMONICS); SHT_ANALYSIS /
 * SHT_ADJOINT_SYNTHESIS read phase and write alm[] (flags SHT_ADD_OUTPUT,
 * SHT_NO_POLAR_OPT, SHT_REAL_HARMONICS).  sht_execute_rings: SHT_SYNTHESIS /
 * SHT_ADJOINT_ANALYSIS read phase (every entry, no polar cut) and write map[]
 * (SHT_ADJOINT_ANALYSIS applies the ring weights; flag SHT_ADD_OUTPUT);
 * SHT_ANALYSIS / SHT_ADJOINT_SYNTHESIS read map[] and write phase.  Both use the
 * plan's workspace like sht_execute (calls sharing a plan must not overlap),
 * allocate nothing and are asynchronous on cuda_stream.  Errors:
 * SHT_ERR_INVALID_ARG (NULL, bad type or flags), SHT_ERR_CUDA.
 */
SHT_API int sht_execute_legendre(sht_plan_t plan, int type, double *const *alm, double *phase, int flags,
                                 void *cuda_stream);
SHT_API int sht_execute_rings(sht_plan_t plan, int type, double *phase, double *const *map, int flags,
                              void *cuda_stream);

/* ---- transforms without allocation -------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory while they run transforms -- code recorded under
 * CUDA stream capture (cudaMalloc / cudaFree cannot be captured and
 * synchronise the device), processes whose GPU memory is held by another
 * allocator's pool, or latency-bound loops that cannot take the implicit
 * device synchronisation of an allocation.
 *
 * sht_execute_noalloc runs the same transform as sht_execute on a plan made
 * beforehand, with the same arguments and results, for the types
 * SHT_SYNTHESIS, SHT_ANALYSIS, SHT_ADJOINT_SYNTHESIS and SHT_ADJOINT_ANALYSIS
 * (SHT_DERIV_SYNTHESIS is rejected with SHT_ERR_INVALID_ARG) and the flags
 * SHT_ADD_OUTPUT, SHT_NO_POLAR_OPT and SHT_REAL_HARMONICS.  Its per-call
 * working memory (the phase array, the analysis partial sums and the converted
 * a_lm tables) comes from a fixed 64 MiB area compiled into the library, and
 * the call allocates nothing, on the device or the host.  What the plan
 * allocated when it was made is still used: its read-only tables and, for
 * rings longer than 14336 points, its FFT scratch slots.  Every GPU that
 * loads the library holds the area until the process exits.  Limit:
 * transforms whose working memory exceeds 64 MiB (about nmaps * nm * npairs *
 * 32 bytes for the phase array, plus the analysis partials) are rejected with
 * SHT_ERR_UNSUPPORTED, the message giving the size needed.  The first call on
 * each device looks up the area's device address (cudaGetSymbolAddress) and
 * keeps it: make that first call before any stream capture begins, and do not
 * call cudaDeviceReset afterwards (the kept address would be stale).  All
 * calls on a device share the one area and it keeps the last call's contents
 * (nothing in it needs to start at zero): calls that overlap on the GPU -- on
 * different streams or from different threads -- race.  The plan's workspace
 * pointers point at the area while the call runs, so no other call on the same
 * plan, sht_execute included, may run concurrently.  No profiling events are
 * recorded.  Errors: as sht_execute, plus SHT_ERR_UNSUPPORTED for the size.
 */
SHT_API int sht_execute_noalloc(sht_plan_t plan, int type, double *const *alm, double *const *map, int flags,
                                void *cuda_stream);

/* ---- batches of independent transforms ----------------------------------------
 * Sect. 3.2 runs several transforms of one plan together; a batch goes further
 * and runs the transforms of many distinct plans -- different lmax, grids,
 * ncomp, spins or precisions -- through the same launches.  The work items of
 * all plans are merged per kernel and ordered longest first, so one grid per
 * stage covers the whole batch and the GPU's block scheduler balances the
 * uneven problems.
 *
 * sht_batch_create takes nplans distinct plans (all made on one device) and
 * builds the merged work lists and per-plan argument records on that device;
 * the batch refers to the plans, which must outlive it.  Limit: the plans'
 * arrays per side, each plan's count rounded up to a power of two, sum to at
 * most 1024 (SHT_ERR_UNSUPPORTED otherwise).  Errors: SHT_ERR_INVALID_ARG
 * (NULL, repeated plan, mixed devices), SHT_ERR_UNSUPPORTED, SHT_ERR_CUDA.
 *
 * sht_batch_execute runs transform `type` of every plan at once on
 * cuda_stream.  alm[k] and map[k] are host arrays holding plan k's device
 * pointers, exactly as sht_execute takes them; flags apply to all plans.
 * Results equal those of sht_execute per plan.  The call neither allocates
 * nor copies nor synchronises (pointers travel as kernel parameters), so it
 * can be captured in a CUDA graph; a captured graph keeps the pointers of the
 * call that was captured.  Each plan runs with the analysis tiling it had
 * when the batch was created.  Each plan's workspace is used, so no plan of the
 * batch may run elsewhere meanwhile, and calls on one batch must not overlap.
 * Errors: SHT_ERR_INVALID_ARG, SHT_ERR_CUDA.
 */
SHT_API int sht_batch_create(int nplans, const sht_plan_t *plans, sht_batch_t *out);
SHT_API int sht_batch_execute(sht_batch_t batch, int type, double *const *const *alm, double *const *const *map,
                              int flags, void *cuda_stream);
/* number of plans in the batch (0 for NULL) */
SHT_API int sht_batch_size(sht_batch_t batch);
SHT_API void sht_batch_destroy(sht_batch_t batch);

/* ---- errors --------------------------------------------------------------- */
SHT_API const char *sht_strerror(int code);
SHT_API const char *sht_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SHT_GB300_H */
