// stages.cu -- the two stages of a transform as separate calls, for the
// distributed decomposition of Sect. 4.2 (Figs. 3 and 4).
//
// A distributed synthesis runs the Legendre stage for the task's own m values
// over every ring, rearranges the phase array F_m(theta_y) among the tasks so
// that each holds all m for its own rings, and runs the ring FFTs there; the
// analysis runs the same steps backwards.  sht_execute_legendre and
// sht_execute_rings are those two stages of a plan's transform, with the phase
// array in caller-owned device memory in a per-ring layout (the plan's internal
// one is per ring pair): phase[c][i][y] is the complex coefficient of map c,
// m = mval[i] (the plan's m list), ring y of the plan's geometry.
#include <string.h>

#include "sht_internal.h"

namespace sht {
namespace {

// user[c][i][y] <- internal[c][i][p][slot]; pairs below the synthesis' first
// written pair (the polar cut) give zero
__global__ void phase_pack(int nmaps, int nm, int npairs, int nrings, const int2 *__restrict__ pair_rings,
                           const int *__restrict__ syn_first, const double2 *__restrict__ in,
                           double2 *__restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, c = blockIdx.z;
  if (p >= npairs) return;
  const int2 r = pair_rings[p];
  const bool cut = syn_first && p < syn_first[i];
  const double2 *src = in + (((size_t)c * nm + i) * npairs + p) * 2;
  double2 *dst = out + ((size_t)c * nm + i) * nrings;
  dst[r.x] = cut ? make_double2(0.0, 0.0) : src[0];
  if (r.y >= 0) dst[r.y] = cut ? make_double2(0.0, 0.0) : src[1];
}

// internal[c][i][p][slot] <- user[c][i][y]
__global__ void phase_unpack(int nmaps, int nm, int npairs, int nrings, const int2 *__restrict__ pair_rings,
                             const double2 *__restrict__ in, double2 *__restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, c = blockIdx.z;
  if (p >= npairs) return;
  const int2 r = pair_rings[p];
  const double2 *src = in + ((size_t)c * nm + i) * nrings;
  double2 *dst = out + (((size_t)c * nm + i) * npairs + p) * 2;
  dst[0] = src[r.x];
  dst[1] = r.y >= 0 ? src[r.y] : make_double2(0.0, 0.0);
}

int check_common(const sht_plan_s *P, int type, int flags, int allowed) {
  if (!P) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
  if (type < SHT_SYNTHESIS || type > SHT_ADJOINT_ANALYSIS) return set_error(SHT_ERR_INVALID_ARG, "bad type %d", type);
  if (flags & ~allowed) return set_error(SHT_ERR_INVALID_ARG, "unknown flags");
  return SHT_OK;
}

}  // namespace
}  // namespace sht

extern "C" int sht_execute_legendre(sht_plan_t P, int type, double *const *alm, double *phase, int flags,
                                    void *stream) {
  using namespace sht;
  int rc = check_common(P, type, flags, SHT_ADD_OUTPUT | SHT_NO_POLAR_OPT | SHT_REAL_HARMONICS);
  if (rc != SHT_OK) return rc;
  if (!alm || !phase) return set_error(SHT_ERR_INVALID_ARG, "pointer arrays are NULL");
  DevPtrs A;
  memset(&A, 0, sizeof(A));
  for (int j = 0; j < P->nmaps; ++j) {
    if (!alm[j]) return set_error(SHT_ERR_INVALID_ARG, "NULL device pointer at index %d", j);
    A.p[j] = alm[j];
  }
  const int per = P->spin ? 2 : 1;
  for (int j = P->nmaps; j < P->nmaps_pad; ++j) A.p[j] = alm[j % per];
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) {
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int polar = (flags & SHT_NO_POLAR_OPT) ? 0 : 1;
  const int add = (flags & SHT_ADD_OUTPUT) ? 1 : 0;
  const bool real = (flags & SHT_REAL_HARMONICS) != 0;
  const int mode = real ? kAlmReal : 0;
  const bool mixed = P->precision == SHT_MIXED;
  const dim3 grid((P->npairs + 127) / 128, P->nm, P->nmaps);
  cudaError_t e = cudaSuccess;
  if (type == SHT_SYNTHESIS || type == SHT_ADJOINT_ANALYSIS) {  // a_lm -> F
    if (add) {
      if (cur != P->device) cudaSetDevice(cur);
      return set_error(SHT_ERR_INVALID_ARG, "SHT_ADD_OUTPUT applies to the a_lm of an analysis-type Legendre stage");
    }
    if (mixed && P->nsyn_lo[polar])
      e = fork_join(
          st, P->side, P->ev_fork, P->ev_join, [&](cudaStream_t s) { return launch_leg_syn_mixed(P, A, polar, s, mode); },
          [&](cudaStream_t s) { return launch_leg_syn_fp64(P, A, polar, s, true, mode); });
    else
      e = mixed ? launch_leg_syn_mixed(P, A, polar, st, mode) : launch_leg_syn_fp64(P, A, polar, st, false, mode);
    if (e == cudaSuccess && P->nm > 0 && P->npairs > 0) {
      phase_pack<<<grid, 128, 0, st>>>(P->nmaps, P->nm, P->npairs, P->nrings, P->d_pair_rings,
                                       P->d_syn_first[polar], P->d_phase, reinterpret_cast<double2 *>(phase));
      e = cudaGetLastError();
    }
  } else {  // G -> a_lm
    if (P->nm > 0 && P->npairs > 0) {
      phase_unpack<<<grid, 128, 0, st>>>(P->nmaps, P->nm, P->npairs, P->nrings, P->d_pair_rings,
                                         reinterpret_cast<const double2 *>(phase), P->d_phase);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      if (mixed && P->nana_lo[polar])
        e = fork_join(
            st, P->side, P->ev_fork, P->ev_join, [&](cudaStream_t s) { return launch_leg_ana_mixed(P, A, polar, s); },
            [&](cudaStream_t s) { return launch_leg_ana_fp64(P, A, polar, s, true); });
      else
        e = mixed ? launch_leg_ana_mixed(P, A, polar, st) : launch_leg_ana_fp64(P, A, polar, st);
    }
    if (e == cudaSuccess) e = launch_ana_reduce(P, A, polar, add, st, real);
  }
  if (cur != P->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return SHT_OK;
}

extern "C" int sht_execute_rings(sht_plan_t P, int type, double *phase, double *const *map, int flags,
                                 void *stream) {
  using namespace sht;
  int rc = check_common(P, type, flags, SHT_ADD_OUTPUT);
  if (rc != SHT_OK) return rc;
  if (!map || !phase) return set_error(SHT_ERR_INVALID_ARG, "pointer arrays are NULL");
  DevPtrs M;
  memset(&M, 0, sizeof(M));
  for (int j = 0; j < P->nmaps; ++j) {
    if (!map[j]) return set_error(SHT_ERR_INVALID_ARG, "NULL device pointer at index %d", j);
    M.p[j] = map[j];
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != P->device) {
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int add = (flags & SHT_ADD_OUTPUT) ? 1 : 0;
  const dim3 grid((P->npairs + 127) / 128, P->nm, P->nmaps);
  cudaError_t e = cudaSuccess;
  if (type == SHT_SYNTHESIS || type == SHT_ADJOINT_ANALYSIS) {  // F -> maps (every pair read: no polar cut)
    if (P->nm > 0 && P->npairs > 0) {
      phase_unpack<<<grid, 128, 0, st>>>(P->nmaps, P->nm, P->npairs, P->nrings, P->d_pair_rings,
                                         reinterpret_cast<const double2 *>(phase), P->d_phase);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_fft_syn(P, M, 0, type == SHT_ADJOINT_ANALYSIS, add, st);
  } else {  // maps -> G
    if (add) {
      if (cur != P->device) cudaSetDevice(cur);
      return set_error(SHT_ERR_INVALID_ARG, "SHT_ADD_OUTPUT applies to the maps of a synthesis-type ring stage");
    }
    e = launch_fft_ana(P, M, type == SHT_ANALYSIS, st);
    if (e == cudaSuccess && P->nm > 0 && P->npairs > 0) {
      phase_pack<<<grid, 128, 0, st>>>(P->nmaps, P->nm, P->npairs, P->nrings, P->d_pair_rings, nullptr, P->d_phase,
                                       reinterpret_cast<double2 *>(phase));
      e = cudaGetLastError();
    }
  }
  if (cur != P->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return SHT_OK;
}
