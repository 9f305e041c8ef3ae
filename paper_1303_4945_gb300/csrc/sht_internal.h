// sht_internal.h -- data structures shared by the translation units of libsht_gb300.
//
// Layout of the device data a plan holds (all in HBM, built once at plan time):
//   pairs      PairDev[npairs]      ring pairs sorted pole -> equator (Sect. 3.3 order)
//   coef       Coef[ncoef64]        recursion coefficients {A, AK, C, 0} per (m, l), Sect. 4.1
//   coef32     float4[2*ncoef]      the same split into FP32 pairs (mixed form)
//   mpre       double2[nm]          start-value prefactor (mantissa, exponent) per m
//   F / G      double2[nmaps][nm][npairs][2]   phase arrays of Eqs. syn2 / ana2 (north, south)
//   part       double[..]           per-tile partial sums of the analysis Legendre stage
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/sht_gb300.h"

namespace sht {

constexpr int kMaxPtr = 32;       // max device pointers per execute (maps or a_lm arrays)
constexpr int kMaxJobs = 16;      // ncomp limit
constexpr int kSynTile = 128;     // ring pairs per synthesis Legendre CTA (one per thread)
constexpr int kAnaThreads = 128;  // threads per analysis Legendre CTA
constexpr int kAnaGroupTiles = 16;  // most tiles a mixed analysis item walks, one after another
constexpr int kAnaItemsPerSm = 24;  // fewest mixed analysis items per SM the grouping leaves
constexpr int kMaxRadix = 8 * 4;  // odd radices with register butterflies and constant cos/sin tables (primes <= 31)
constexpr int kMaxBigRadix = 127;  // odd radices above 31 run as shared-memory sweeps (fft_stage_big)
constexpr int kFftThreads = 512;
constexpr int kFftMinBlocks = 512 / kFftThreads;  // launch bound: at most 128 registers a thread
// longest in-place transform: the ring buffer (16 bytes a point) must fit the
// opt-in shared memory of one CTA (227 KB on sm_103a)
constexpr int kFftMaxLen = 14336;
constexpr double kFp64PolarCap = 0.05;  // rad; see sht_plan_s::fp64_m_below
// longest transform at all: longer rings run from a global scratch slot per CTA
// (1 MiB each), which stays in L2
constexpr int kFftMaxGlobalLen = 65536;

// Extended exponent of the FP64 recursion: a pair (lambda_{l-1}, lambda_l) is
// stored as value * 2^(kScaleStep * scale); it contributes only at scale 0.
constexpr int kScaleStep = 600;
constexpr double kScaleUp = 0x1p+300;     // rescale when |lambda| exceeds this
constexpr double kScaleFactor = 0x1p-600;

struct PairDev {
  double x;        // cos(theta) of the ring in the north slot (libm cos of the given theta)
  double l1_hi;    // log2(sin theta), double-double
  double l1_lo;
  double l2_hi;    // log2(tan(theta/2)), double-double
  double l2_lo;
  int pole;        // 1 if theta == 0 exactly (sin theta == 0)
  int south;       // 1 if the pair has a mirrored southern ring
};

// Per-ring data for the FFT stage.
struct RingDev {
  int64_t ofs;
  int nphi;
  int stride;
  double phi0;
  double weight;
};

struct FftPlanDev {
  int n;          // ring length
  int kind;       // 0 mixed radix, 1 Rader, 2 Bluestein
  int len;        // inner transform length (n, n-1 or the Bluestein size)
  int nrad;
  int rad[24];
  const double2 *w;      // twiddles e^{-2 pi i k / len}, k < len
  const int *pos;        // plain: position of X_k after the DIF passes (digit reversal)
  const int *perm_in;    // Rader: g^q mod n
  const int *inv_out;    // Rader: index p with g^{-p} = k, for k = 1..n-1
  const double2 *spec;   // Rader / Bluestein kernel spectrum (1/len folded in)
  const double2 *chirp;  // Bluestein: e^{-pi i k^2 / n}
  // the same three tables as hi/lo float pairs (re.h, re.l, im.h, im.l) for the
  // double-float engine of mixed plans (null in FP64 plans)
  const float4 *wf, *specf, *chirpf;
};

struct DevPtrs {
  double *p[kMaxPtr];
};

// device pointers of every plan of a batch, passed by value to the batched kernels
constexpr int kMaxBatchPtr = 1024;
struct PtrTable {
  double *p[kMaxBatchPtr];
};

// recursion coefficients of one (m, l): lambda_{l+1} = (a x + ak) lambda_l - c lambda_{l-1}
struct __align__(32) Coef {
  double a, ak, c, pad;
};

}  // namespace sht

// ----------------------------------------------------------------------------
// Opaque handles of the C ABI.
// ----------------------------------------------------------------------------
struct sht_geom_s {
  int nrings = 0;
  std::vector<double> theta, phi0, weight;
  std::vector<int> nphi, stride;
  std::vector<int64_t> ofs;
};

struct sht_alm_s {
  int lmax = 0, mmax = 0, nm = 0, stride = 1;
  std::vector<int> mval;
  std::vector<int64_t> mstart;
};

struct sht_plan_s {
  int device = 0;
  int sms = 1;  // multiprocessors of the device
  int lmax = 0, mmax = 0, nm = 0, astride = 1, spin = 0, ncomp = 0, precision = 0;
  int nmaps = 0;      // arrays per side (ncomp, or 2 ncomp for spin)
  int njobs_pad = 1;  // ncomp rounded up to a power of two (kernel template size)
  int nmaps_pad = 1;  // arrays per side for njobs_pad jobs
  int nrings = 0, npairs = 0;
  std::vector<int> mval;
  std::vector<int64_t> mstart;
  std::vector<int> pair_n, pair_s;         // ring index of the north / south slot (-1 none)
  std::vector<double> pair_pole;           // per pair: distance of its rings from the nearer pole (rad)
  std::vector<int> first_pair;             // per m: first pair not removed by the polar cut
  std::vector<int64_t> coef_off;           // per m: table index of l = l0
  int64_t ncoef = 0;
  // entries of the FP64 tables (coef, and d_pm64 per array): all of them for an FP64
  // plan; for a mixed plan the prefix its FP64 columns read (m < the FP64 column bound)
  int64_t ncoef64 = 0;

  // device arrays
  sht::PairDev *d_pairs = nullptr;
  int2 *d_pair_rings = nullptr;
  sht::RingDev *d_rings = nullptr;
  int *d_mval = nullptr;
  int64_t *d_mstart = nullptr;
  int64_t *d_coef_off = nullptr;
  sht::Coef *d_coef = nullptr;
  float4 *d_coef32 = nullptr;
  float4 *d_alm32 = nullptr;               // mixed form: a_lm as double-float pairs [array][ncoef]
  double2 *d_pm64 = nullptr;               // FP64 spin form: P = E + iB, M = E - iB [array][ncoef64]
  double2 *d_mpre = nullptr;
  int *d_minv = nullptr;                   // m -> index in mval, or -1
  double2 *d_phase = nullptr;              // F / G workspace
  double *d_part = nullptr;                // analysis partials
  int64_t part_doubles = 0;

  // work lists (polar-cut / uncut): synthesis (mi, first pair) and analysis (mi, tile, part offset)
  int2 *d_syn_items[2] = {nullptr, nullptr};
  int nsyn_items[2] = {0, 0};
  int *d_syn_first[2] = {nullptr, nullptr};  // per m: first pair the synthesis wrote (FFT reads 0 below)
  int4 *d_ana_items[2] = {nullptr, nullptr};
  int nana_items[2] = {0, 0};
  int64_t *d_ana_part_off[2] = {nullptr, nullptr};  // per m
  int *d_ana_nslot[2] = {nullptr, nullptr};         // per m: partial-sum slots (one per item)
  int ana_ppt = 4;                                  // ring pairs per analysis thread (tiling)
  int batch_refs = 0;                               // batches built on this plan's work lists
  // host copies of the work lists with their costs (l count x pairs), for merging into batches
  std::vector<std::pair<int64_t, int2>> syn_list[2];
  std::vector<std::pair<int64_t, int4>> ana_list[2];
  // mixed form: the work items of columns m < fp64_m_below that touch a ring within
  // kFp64PolarCap of a pole run in the FP64 kernels (work lists of their own): there
  // the small-m recursion is non-oscillatory for l < ~1/theta and amplifies its
  // per-step rounding by a power of l
  int fp64_m_below = 0;
  bool fft_df = false;  // ring FFTs in double-float (mixed plans, by default)
  // mixed plans: the synthesis contraction on the tensor cores (legendre_tc.cu)
  int tc_syn = 0;
  // mixed plans: the analysis contraction on the tensor cores (legendre_tc_ana.cu;
  // tiles of kAnaThreads ring pairs, one per thread)
  int tc_ana = 0;
  float tc_lam_bound = 0.f;  // power of two bounding |Lambda_lm| for lmax
  int *d_err = nullptr;      // device status word written by kernels with bounded waits
  float4 *d_join = nullptr;  // mixed plans: join record per (m index, pair), 3 float4 each
  int64_t triples_joined = 0;  // steps from each kept pair's join block on (polar cut applied)
  int m_identity = 0;   // the m list is 0, 1, ..., nm - 1
  // the FP64 columns run beside the mixed kernels: a side stream forked and joined by events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  cudaEvent_t ev_lo = nullptr;
  int2 *d_syn_lo[2] = {nullptr, nullptr};
  int nsyn_lo[2] = {0, 0};
  int4 *d_ana_lo[2] = {nullptr, nullptr};
  int nana_lo[2] = {0, 0};
  std::vector<std::pair<int64_t, int2>> syn_list_lo[2];
  std::vector<std::pair<int64_t, int4>> ana_list_lo[2];
  int64_t triples[2] = {0, 0};

  // FFT
  std::vector<void *> fft_allocs;
  sht::FftPlanDev *d_fft = nullptr;
  int nfft = 0;
  int *d_pair_fft = nullptr;  // per pair: plan index
  int fft_smem = 0;           // bytes of dynamic shared memory for the FFT kernels
  std::vector<int> pair_len;  // per pair: the longer ring length (FFT cost)
  double2 *d_fft_scratch = nullptr;  // rings beyond kFftMaxLen: one slot of fft_slot_len points per CTA
  int fft_slots = 0, fft_slot_len = 0;

  int64_t workspace = 0;

  // measurement: event pairs around each launch while profiling is on
  int prof_on = 0;
  struct ProfRec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof;
};

// ----------------------------------------------------------------------------
// Cross-TU launch helpers (all return cudaError_t of the launch).
// ----------------------------------------------------------------------------
namespace sht {
constexpr int kAlmDeriv = 1, kAlmReal = 2, kAlmHalf = 4;  // a_lm conversion modes (see launch_alm_prepare_fp64)

// Runs side_fn on stream `side` concurrently with main_fn on `st`: `side` waits for
// the work queued on `st` so far, side_fn is launched first (its CTAs are the
// long ones), and `st` waits for it before anything queued later.  The pattern
// is capturable in a CUDA graph.
template <class MainFn, class SideFn>
inline cudaError_t fork_join(cudaStream_t st, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join,
                             MainFn &&main_fn, SideFn &&side_fn) {
  cudaError_t e = cudaEventRecord(fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
  if (e != cudaSuccess) return e;
  cudaError_t es = side_fn(side);
  e = cudaEventRecord(join, side);
  cudaError_t em = main_fn(st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join, 0);
  if (es != cudaSuccess) return es;
  if (em != cudaSuccess) return em;
  return e;
}

// records a message for sht_last_error() on this thread and returns code
int set_error(int code, const char *fmt, ...);
// plan-time tables
cudaError_t launch_coef_tables(const sht_plan_s *P, cudaStream_t st);
cudaError_t launch_fft_spectrum(const FftPlanDev *host_plan, const FftPlanDev *dev_plan,
                                const double2 *src, double2 *dst, int len, double scale,
                                cudaStream_t st);
// Legendre stage
// lo: run the mixed plan's FP64 columns (work lists d_syn_lo / d_ana_lo)
cudaError_t launch_leg_syn_fp64(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st,
                                bool lo = false, int mode = 0);
cudaError_t launch_leg_ana_fp64(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st,
                                bool lo = false);
// grad: the gradient factor of Sect. 4.5's adjoint for the stored m >= 0 a_lm (m > 0 doubled)
cudaError_t launch_ana_reduce(const sht_plan_s *P, const DevPtrs &alm, int polar, int add, cudaStream_t st,
                              bool real = false, bool grad = false);
cudaError_t launch_leg_syn_mixed(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st, int mode = 0);
// the Legendre stage over an explicit work list (stage 0 synthesis, 1 analysis), no a_lm conversion
// amode: kAlmReal / kAlmHalf bits for the spin-0 synthesis, which reads the a_lm directly
cudaError_t launch_leg_fp64_items(const sht_plan_s *P, int stage, const DevPtrs &alm, int polar, const void *items,
                                  int n, cudaStream_t st, int amode = 0);
cudaError_t launch_leg_mixed_items(const sht_plan_s *P, int stage, int polar, const void *items, int n,
                                   cudaStream_t st);
cudaError_t launch_leg_ana_mixed(const sht_plan_s *P, const DevPtrs &alm, int polar, cudaStream_t st);
// tensor-core synthesis (legendre_tc.cu): mixargs is the mixed kernels' argument
// record (MixArgs) with its synthesis work list set; n work items
cudaError_t launch_leg_tc_syn(const sht_plan_s *P, const void *mixargs, int n, cudaStream_t st);
cudaError_t tc_prepare_device();
cudaError_t launch_join_records(const sht_plan_s *P, cudaStream_t st);
// batches: one TcArgs record per plan of a tensor-core group
size_t tc_args_size();
void leg_tc_fill_args(const sht_plan_s *P, int polar, int ptr_off, void *out);
cudaError_t launch_leg_tc_batch(int spin, int nj, const void *targs, const int4 *items, int n, cudaStream_t st);
bool tc_supported(int spin, int njobs_pad);
float tc_lambda_bound(int lmax);
// tensor-core analysis (legendre_tc_ana.cu): mixargs with its analysis work list set
cudaError_t launch_leg_tc_ana(const sht_plan_s *P, const void *mixargs, int n, cudaStream_t st);
// batches: one TcArgs record per plan of a tensor-core analysis group
cudaError_t launch_leg_tc_ana_batch(int spin, int nj, const void *targs, const int4 *items, int n, cudaStream_t st);
cudaError_t tc_ana_prepare_device();
bool tc_ana_supported(int spin, int njobs_pad);
// ring FFTs
// ring pairs [p0, p1) (p1 < 0: to the last pair)
cudaError_t launch_fft_syn(const sht_plan_s *P, const DevPtrs &map, int polar, int weighted, int add,
                           cudaStream_t st, int p0 = 0, int p1 = -1);
cudaError_t launch_fft_ana(const sht_plan_s *P, const DevPtrs &map, int weighted, cudaStream_t st, int p0 = 0,
                           int p1 = -1);
// lets every FFT kernel use the device's opt-in shared memory (once per device, at plan time:
// the limit is one value per kernel and process, so it is only ever raised, never per call)
cudaError_t fft_prepare_device(int device);

// batches: per-plan argument records (copied to the device once, at batch creation) and
// launches over merged work lists; item.w selects the record, PtrTable holds the caller's
// arrays, each plan's from record.ptr_off on
size_t leg_fp64_args_size();
size_t leg_mixed_args_size();
size_t fft_args_size();
void leg_fp64_fill_args(const sht_plan_s *P, int polar, int ptr_off, void *out, bool lo = false);
void leg_mixed_fill_args(const sht_plan_s *P, int polar, int ptr_off, void *out);
void fft_fill_args(const sht_plan_s *P, int polar, int weighted, int add, int ptr_off, void *out);
// a_lm -> the P = E+iB / M = E-iB tables (FP64 spin) or double-float tables (mixed); mode bits:
// kAlmDeriv, the first-derivative mode of Sect. 4.3 (spin-1 plan, E = sqrt(l(l+1)) a of ncomp
// spin-0 arrays, B = 0); kAlmReal, inputs in real-harmonic storage; kAlmHalf, the m > 0
// coefficients halved (the adjoint analysis of a gradient, see SHT_GRADIENT)
cudaError_t launch_alm_prepare_fp64(const sht_plan_s *P, const DevPtrs &alm, cudaStream_t st, int mode = 0);
cudaError_t launch_alm_prepare_mixed(const sht_plan_s *P, const DevPtrs &alm, cudaStream_t st, int mode = 0);
// stage 0: synthesis, 1: analysis
cudaError_t launch_leg_fp64_batch(int stage, int spin, int nj, int ppt, const void *args, const int4 *items,
                                  int n, const PtrTable &tbl, cudaStream_t st);
cudaError_t launch_leg_mixed_batch(int stage, int spin, int nj, int ppt, const void *args, const int4 *items,
                                   int n, const PtrTable &tbl, cudaStream_t st);
cudaError_t launch_fft_batch(int stage, bool df, const void *args, const int4 *items, int n, int smem,
                             const PtrTable &tbl, cudaStream_t st);
}  // namespace sht
