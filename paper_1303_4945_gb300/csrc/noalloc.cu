// noalloc.cu -- sht_execute_noalloc: a transform that allocates nothing.
//
// Some callers may not allocate device memory while they run transforms:
// code recorded under CUDA stream capture (cudaMalloc / cudaFree are not
// capturable and synchronise the device), processes whose GPU memory is
// reserved by another allocator's pool, or latency-bound loops that cannot
// afford the implicit device synchronisation of cudaMalloc / cudaFree.
// This entry point runs the transform of an existing plan exactly like
// sht_execute, but takes its per-call working memory -- the phase array F/G,
// the analysis tile sums and the converted a_lm tables (both, for a mixed plan
// with FP64 columns) -- from one fixed area compiled into the library
// (kNoallocBytes below), so the call itself makes no allocation of any kind.
// Two things still come from the plan, both allocated once when the plan was
// made: its read-only tables (recursion coefficients, ring pairs, work lists,
// FFT twiddles) and, for rings longer than the in-shared-memory limit
// (kFftMaxLen points), its FFT scratch slots.  The plan's workspace pointers
// are swapped to the area for the length of the call and restored on return,
// so no other call on the same plan (sht_execute included) may run
// concurrently from another thread.  Every GPU that loads the library holds
// the area until the process exits.
//
// The area is shared by every call on a device and keeps whatever the last
// call left in it; the kernels write every element they later read (no part
// of it has to start at zero).  Calls that overlap on the GPU -- on
// different streams, or from different threads -- race on the area.
// The area's device address is looked up once per device and kept:
// cudaDeviceReset is not supported once the call has been used on a device
// (a reset can move the area, and the kept address would then be stale).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "sht_internal.h"

namespace {

constexpr int64_t kNoallocBytes = int64_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_area[kNoallocBytes];

// device address of g_noalloc_area per device (the host-side symbol is not one)
void *g_area_addr[kMaxDevices] = {};
std::mutex g_area_mu;

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int sht_execute_noalloc(sht_plan_t P, int type, double *const *alm, double *const *map, int flags,
                                   void *stream) {
  using namespace sht;
  if (!P) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (type < SHT_SYNTHESIS || type > SHT_ADJOINT_ANALYSIS) return set_error(SHT_ERR_INVALID_ARG, "bad type %d", type);
  if (flags & ~(SHT_ADD_OUTPUT | SHT_NO_POLAR_OPT | SHT_REAL_HARMONICS))
    return set_error(SHT_ERR_INVALID_ARG, "unknown flags");
  const bool real = (flags & SHT_REAL_HARMONICS) != 0;
  const int mode = real ? kAlmReal : 0;
  if (!alm || !map) return set_error(SHT_ERR_INVALID_ARG, "pointer arrays are NULL");
  if (P->device < 0 || P->device >= kMaxDevices) return set_error(SHT_ERR_UNSUPPORTED, "device index too large");
  DevPtrs A, M;
  memset(&A, 0, sizeof(A));
  memset(&M, 0, sizeof(M));
  for (int j = 0; j < P->nmaps; ++j) {
    if (!alm[j] || !map[j]) return set_error(SHT_ERR_INVALID_ARG, "NULL device pointer at index %d", j);
    A.p[j] = alm[j];
    M.p[j] = map[j];
  }
  const int per = P->spin ? 2 : 1;
  for (int j = P->nmaps; j < P->nmaps_pad; ++j) A.p[j] = alm[j % per];

  // per-call working memory, carved from the static area
  const bool synth = (type == SHT_SYNTHESIS || type == SHT_ADJOINT_ANALYSIS);
  const bool mixed = P->precision == SHT_MIXED;
  const int64_t b_phase = align256((int64_t)P->nmaps_pad * P->nm * P->npairs * 2 * (int64_t)sizeof(double2));
  const int64_t b_part = synth ? 0 : align256(P->part_doubles * (int64_t)sizeof(double));
  const int64_t b_alm32 = (synth && mixed) ? align256(P->ncoef * P->nmaps_pad * (int64_t)sizeof(float4)) : 0;
  const bool lo = mixed && (P->nsyn_lo[0] || P->nsyn_lo[1]);  // mixed plan with FP64 columns
  const int64_t b_pm64 =
      (synth && P->spin && (!mixed || lo)) ? align256(P->ncoef64 * P->nmaps_pad * (int64_t)sizeof(double2)) : 0;
  const int64_t need = b_phase + b_part + b_alm32 + b_pm64;
  if (need > kNoallocBytes)
    return set_error(SHT_ERR_UNSUPPORTED, "this transform needs %lld bytes of working memory; the static area holds %lld",
                     (long long)need, (long long)kNoallocBytes);

  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) {
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  }
  // one-time set-up per device (with that device current): the device address of the area
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_area_mu);
    if (!g_area_addr[P->device]) {
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_area);
      if (e != cudaSuccess) {
        if (cur != P->device) cudaSetDevice(cur);
        return set_error(SHT_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      }
      g_area_addr[P->device] = ptr;
    }
    base = static_cast<unsigned char *>(g_area_addr[P->device]);
  }

  // run the plan's kernels on the area: swap the workspace pointers in and back
  // out (calls that share a plan must not overlap, as for sht_execute)
  double2 *phase0 = P->d_phase;
  double *part0 = P->d_part;
  float4 *alm320 = P->d_alm32;
  double2 *pm640 = P->d_pm64;
  P->d_phase = reinterpret_cast<double2 *>(base);
  if (b_part) P->d_part = reinterpret_cast<double *>(base + b_phase);
  if (b_alm32) P->d_alm32 = reinterpret_cast<float4 *>(base + b_phase);
  if (b_pm64) P->d_pm64 = reinterpret_cast<double2 *>(base + b_phase + b_alm32);
  cudaStream_t st = (cudaStream_t)stream;
  const int polar = (flags & SHT_NO_POLAR_OPT) ? 0 : 1;
  const int add = (flags & SHT_ADD_OUTPUT) ? 1 : 0;
  cudaError_t e;
  if (synth) {
    if (mixed && P->nsyn_lo[polar])  // FP64 columns beside the mixed kernel
      e = fork_join(
          st, P->side, P->ev_fork, P->ev_join, [&](cudaStream_t s) { return launch_leg_syn_mixed(P, A, polar, s, mode); },
          [&](cudaStream_t s) { return launch_leg_syn_fp64(P, A, polar, s, true, mode); });
    else
      e = mixed ? launch_leg_syn_mixed(P, A, polar, st, mode) : launch_leg_syn_fp64(P, A, polar, st, false, mode);
    if (e == cudaSuccess) e = launch_fft_syn(P, M, polar, type == SHT_ADJOINT_ANALYSIS, add, st);
  } else {
    e = launch_fft_ana(P, M, type == SHT_ANALYSIS, st);
    if (e == cudaSuccess) {
      if (mixed && P->nana_lo[polar])
        e = fork_join(
            st, P->side, P->ev_fork, P->ev_join, [&](cudaStream_t s) { return launch_leg_ana_mixed(P, A, polar, s); },
            [&](cudaStream_t s) { return launch_leg_ana_fp64(P, A, polar, s, true); });
      else
        e = mixed ? launch_leg_ana_mixed(P, A, polar, st) : launch_leg_ana_fp64(P, A, polar, st);
    }
    if (e == cudaSuccess) e = launch_ana_reduce(P, A, polar, add, st, real, false);
  }
  P->d_phase = phase0;
  P->d_part = part0;
  P->d_alm32 = alm320;
  P->d_pm64 = pm640;
  if (cur != P->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return SHT_OK;
}
