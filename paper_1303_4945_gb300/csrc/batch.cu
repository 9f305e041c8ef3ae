// batch.cu -- sht_batch_execute: the transforms of many plans in merged launches.
//
// A batch is a fixed list of distinct plans on one device, built once.  At
// creation the work items of all plans (synthesis tiles (m, first pair),
// analysis tiles (m, pair tile), ring-pair FFTs (pair, map)) are merged into
// one list per kernel and sorted by cost, longest first, so each stage of the
// whole batch is one grid: the block scheduler hands CTAs out in index order
// as SMs free up, i.e. greedy longest-processing-time list scheduling over the
// uneven problems.  Plans whose Legendre kernels differ (precision, spin
// class, padded job count, analysis tiling, synthesis or analysis on the tensor
// cores or not) form separate groups, one launch each; every item
// carries the index of its plan's argument record, which lives on the device
// from creation on.  Per call only the caller's array pointers change; they
// travel in the kernel parameters (PtrTable), so an execute neither
// allocates, copies nor synchronises and can be captured in a CUDA graph.
// The per-plan pre- and post-processing (a_lm conversion before synthesis,
// the reduction of analysis tile sums) runs as one small launch per plan.
// Every plan keeps using its own workspace, so the plans of a batch must be
// distinct, and a plan must not run elsewhere while its batch runs; a plan
// cannot change its tiling while a batch refers to it.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <set>

#include "sht_internal.h"

namespace {

struct Group {
  int precision = 0, spin = 0, nj = 1, ppt = 2;
  bool tc = false;                   // mixed plans whose synthesis runs on the tensor cores
  bool tca = false;                  // mixed plans whose analysis runs on the tensor cores
  void *d_targs[2] = {nullptr, nullptr};  // per polar: their TcArgs records (tensor-core kernels)
  std::vector<int> plans;            // batch indices; item.w is the position in this list
  std::vector<char> lo;              // per entry: the mixed plan's FP64 columns (FP64 group)
  void *d_args[2] = {nullptr, nullptr};  // per polar: one argument record per plan
  int4 *d_syn[2] = {nullptr, nullptr};
  int nsyn[2] = {0, 0};
  int4 *d_ana[2] = {nullptr, nullptr};
  int nana[2] = {0, 0};
};

}  // namespace

struct sht_batch_s {
  int device = 0;
  std::vector<sht_plan_s *> plans;
  std::vector<int> ptr_off;  // per plan: first slot of its arrays in the pointer tables
  std::vector<Group> groups;
  void *d_fft_syn[2][2][2] = {};  // [polar][weighted][add]: FFT argument records
  void *d_fft_ana[2] = {};        // [weighted]
  int4 *d_fft_items[2] = {};      // (pair, map, -, plan) by FFT engine: FP64 [0], double-float [1]
  int nfft_items[2] = {};
  int fft_smem = 0;
  std::vector<void *> allocs;
  // FP64 groups run beside mixed groups: a side stream forked and joined by events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

using sht::set_error;

void free_batch(sht_batch_s *B) {
  for (void *p : B->allocs) cudaFree(p);
  if (B->side) cudaStreamDestroy(B->side);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->ev_join) cudaEventDestroy(B->ev_join);
  delete B;
}

template <class T>
cudaError_t upload(sht_batch_s *B, const T *src, size_t count, T **dst) {
  *dst = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, count * sizeof(T));
  if (e != cudaSuccess) return e;
  B->allocs.push_back(*dst);
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t upload_bytes(sht_batch_s *B, const std::vector<unsigned char> &src, void **dst) {
  unsigned char *d = nullptr;
  cudaError_t e = upload(B, src.data(), src.size(), &d);
  *dst = d;
  return e;
}

template <class Item>
void sort_by_cost(std::vector<std::pair<int64_t, Item>> &v) {
  std::stable_sort(v.begin(), v.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
}

template <class Item>
std::vector<Item> strip(const std::vector<std::pair<int64_t, Item>> &v) {
  std::vector<Item> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].second;
  return out;
}

int build(sht_batch_s *B) {
  using namespace sht;
  const int n = (int)B->plans.size();
  // pointer-table slots
  int slots = 0;
  for (int k = 0; k < n; ++k) {
    B->ptr_off.push_back(slots);
    slots += B->plans[k]->nmaps_pad;
  }
  if (slots > kMaxBatchPtr)
    return set_error(SHT_ERR_UNSUPPORTED, "a batch holds at most %d arrays per side (padded); this one needs %d",
                     kMaxBatchPtr, slots);
  // Legendre groups; a mixed plan with FP64 columns is also an entry of an FP64 group
  auto join = [&](int k, int precision, bool lo) {
    const sht_plan_s *P = B->plans[k];
    const int spin_class = P->spin ? 1 : 0;
    const bool tc = precision == SHT_MIXED && P->tc_syn;
    const bool tca = precision == SHT_MIXED && P->tc_ana;
    Group *g = nullptr;
    for (auto &c : B->groups)
      if (c.precision == precision && c.spin == spin_class && c.nj == P->njobs_pad && c.ppt == P->ana_ppt &&
          c.tc == tc && c.tca == tca)
        g = &c;
    if (!g) {
      B->groups.emplace_back();
      g = &B->groups.back();
      g->precision = precision;
      g->spin = spin_class;
      g->nj = P->njobs_pad;
      g->ppt = P->ana_ppt;
      g->tc = tc;
      g->tca = tca;
    }
    g->plans.push_back(k);
    g->lo.push_back(lo ? 1 : 0);
  };
  for (int k = 0; k < n; ++k) {
    const sht_plan_s *P = B->plans[k];
    join(k, P->precision, false);
    if (P->precision == SHT_MIXED && (P->nsyn_lo[0] || P->nsyn_lo[1] || P->nana_lo[0] || P->nana_lo[1]))
      join(k, SHT_FP64, true);
  }
  cudaError_t e = cudaSuccess;
  for (auto &g : B->groups) {
    const bool mixed = g.precision == SHT_MIXED;
    const size_t rec = mixed ? leg_mixed_args_size() : leg_fp64_args_size();
    for (int polar = 0; polar < 2; ++polar) {
      std::vector<unsigned char> args(rec * g.plans.size());
      const bool tcrec = g.tc || g.tca;
      std::vector<unsigned char> targs(tcrec ? tc_args_size() * g.plans.size() : 0);
      std::vector<std::pair<int64_t, int4>> syn, ana;
      for (size_t i = 0; i < g.plans.size(); ++i) {
        const int k = g.plans[i];
        const bool lo = g.lo[i] != 0;
        const sht_plan_s *P = B->plans[k];
        if (mixed)
          leg_mixed_fill_args(P, polar, B->ptr_off[k], args.data() + i * rec);
        else
          leg_fp64_fill_args(P, polar, B->ptr_off[k], args.data() + i * rec, lo);
        if (tcrec) leg_tc_fill_args(P, polar, B->ptr_off[k], targs.data() + i * tc_args_size());
        for (auto &it : (lo ? P->syn_list_lo : P->syn_list)[polar])
          syn.push_back({it.first, make_int4(it.second.x, it.second.y, 0, (int)i)});
        for (auto &it : (lo ? P->ana_list_lo : P->ana_list)[polar])
          ana.push_back({it.first, make_int4(it.second.x, it.second.y, it.second.z, (int)i)});
      }
      sort_by_cost(syn);
      sort_by_cost(ana);
      auto si = strip(syn), ai = strip(ana);
      g.nsyn[polar] = (int)si.size();
      g.nana[polar] = (int)ai.size();
      if (e == cudaSuccess) e = upload_bytes(B, args, &g.d_args[polar]);
      if (e == cudaSuccess && tcrec) e = upload_bytes(B, targs, &g.d_targs[polar]);
      if (e == cudaSuccess) e = upload(B, si.data(), si.size(), &g.d_syn[polar]);
      if (e == cudaSuccess) e = upload(B, ai.data(), ai.size(), &g.d_ana[polar]);
    }
  }
  // FFT records and items
  const size_t rec = fft_args_size();
  for (int polar = 0; polar < 2; ++polar)
    for (int w = 0; w < 2; ++w)
      for (int add = 0; add < 2; ++add) {
        std::vector<unsigned char> args(rec * n);
        for (int k = 0; k < n; ++k) fft_fill_args(B->plans[k], polar, w, add, B->ptr_off[k], args.data() + k * rec);
        if (e == cudaSuccess) e = upload_bytes(B, args, &B->d_fft_syn[polar][w][add]);
      }
  for (int w = 0; w < 2; ++w) {
    std::vector<unsigned char> args(rec * n);
    for (int k = 0; k < n; ++k) fft_fill_args(B->plans[k], 1, w, 0, B->ptr_off[k], args.data() + k * rec);
    if (e == cudaSuccess) e = upload_bytes(B, args, &B->d_fft_ana[w]);
  }
  std::vector<std::pair<int64_t, int4>> fi[2];  // by engine: FP64, double-float
  for (int k = 0; k < n; ++k) {
    const sht_plan_s *P = B->plans[k];
    B->fft_smem = std::max(B->fft_smem, P->fft_smem);
    const int df = P->fft_df ? 1 : 0;
    for (int p = 0; p < P->npairs; ++p)
      for (int j = 0; j < P->nmaps; ++j) fi[df].push_back({(int64_t)P->pair_len[p], make_int4(p, j, 0, k)});
  }
  for (int df = 0; df < 2; ++df) {
    sort_by_cost(fi[df]);
    auto fv = strip(fi[df]);
    B->nfft_items[df] = (int)fv.size();
    if (e == cudaSuccess && !fv.empty()) e = upload(B, fv.data(), fv.size(), &B->d_fft_items[df]);
  }
  int least = 0, greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&B->side, cudaStreamNonBlocking, greatest);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));
  return SHT_OK;
}

}  // namespace

extern "C" int sht_batch_create(int nplans, const sht_plan_t *plans, sht_batch_t *out) {
  using namespace sht;
  if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nplans < 1 || !plans) return set_error(SHT_ERR_INVALID_ARG, "a batch needs at least one plan");
  std::set<const sht_plan_s *> seen;
  for (int k = 0; k < nplans; ++k) {
    if (!plans[k]) return set_error(SHT_ERR_INVALID_ARG, "plan %d is NULL", k);
    if (!seen.insert(plans[k]).second) return set_error(SHT_ERR_INVALID_ARG, "plan %d appears twice", k);
    if (plans[k]->d_fft_scratch)
      return set_error(SHT_ERR_UNSUPPORTED, "plan %d has rings longer than %d points; run it with sht_execute", k,
                       kFftMaxLen);
    if (plans[k]->device != plans[0]->device)
      return set_error(SHT_ERR_INVALID_ARG, "plan %d lives on device %d, plan 0 on device %d", k, plans[k]->device,
                       plans[0]->device);
  }
  auto *B = new sht_batch_s;
  B->device = plans[0]->device;
  B->plans.assign(plans, plans + nplans);
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != B->device) cudaSetDevice(B->device);
  const int rc = build(B);
  if (cur != B->device) cudaSetDevice(cur);
  if (rc != SHT_OK) {
    free_batch(B);
    return rc;
  }
  for (auto *P : B->plans) ++P->batch_refs;
  *out = B;
  return SHT_OK;
}

extern "C" void sht_batch_destroy(sht_batch_t B) {
  if (!B) return;
  int cur = -1;
  const int dev = B->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  for (auto *P : B->plans) --P->batch_refs;
  free_batch(B);
  if (cur != dev) cudaSetDevice(cur);
}

extern "C" int sht_batch_size(sht_batch_t B) { return B ? (int)B->plans.size() : 0; }

extern "C" int sht_batch_execute(sht_batch_t B, int type, double *const *const *alm, double *const *const *map,
                                 int flags, void *stream) {
  using namespace sht;
  if (!B) return set_error(SHT_ERR_INVALID_ARG, "batch is NULL");
  if (type < SHT_SYNTHESIS || type > SHT_ADJOINT_ANALYSIS) return set_error(SHT_ERR_INVALID_ARG, "bad type %d", type);
  if (flags & SHT_REAL_HARMONICS)
    return set_error(SHT_ERR_UNSUPPORTED, "real-harmonic storage is not supported in batches");
  if (flags & ~(SHT_ADD_OUTPUT | SHT_NO_POLAR_OPT)) return set_error(SHT_ERR_INVALID_ARG, "unknown flags");
  if (!alm || !map) return set_error(SHT_ERR_INVALID_ARG, "pointer arrays are NULL");
  const int n = (int)B->plans.size();
  PtrTable TA, TM;
  memset(&TA, 0, sizeof(TA));
  memset(&TM, 0, sizeof(TM));
  std::vector<DevPtrs> A(n), M(n);
  for (int k = 0; k < n; ++k) {
    const sht_plan_s *P = B->plans[k];
    if (!alm[k] || !map[k]) return set_error(SHT_ERR_INVALID_ARG, "pointer list of plan %d is NULL", k);
    memset(&A[k], 0, sizeof(DevPtrs));
    memset(&M[k], 0, sizeof(DevPtrs));
    for (int j = 0; j < P->nmaps; ++j) {
      if (!alm[k][j] || !map[k][j]) return set_error(SHT_ERR_INVALID_ARG, "NULL device pointer: plan %d, array %d", k, j);
      A[k].p[j] = alm[k][j];
      M[k].p[j] = map[k][j];
    }
    const int per = P->spin ? 2 : 1;
    for (int j = P->nmaps; j < P->nmaps_pad; ++j) A[k].p[j] = alm[k][j % per];
    for (int j = 0; j < P->nmaps_pad; ++j) {
      TA.p[B->ptr_off[k] + j] = A[k].p[j];
      TM.p[B->ptr_off[k] + j] = M[k].p[j < P->nmaps ? j : 0];
    }
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != B->device) {
    cudaError_t e = cudaSetDevice(B->device);
    if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int polar = (flags & SHT_NO_POLAR_OPT) ? 0 : 1;
  const int add = (flags & SHT_ADD_OUTPUT) ? 1 : 0;
  cudaError_t e = cudaSuccess;
  // Legendre stage of every group; FP64 groups beside mixed ones when both exist
  auto legendre = [&](int stage) -> cudaError_t {
    bool has[2] = {false, false};
    for (auto &g : B->groups) has[g.precision == SHT_MIXED ? 1 : 0] = true;
    auto run = [&](bool mixed_groups, cudaStream_t s) -> cudaError_t {
      cudaError_t r = cudaSuccess;
      for (auto &g : B->groups) {
        if ((g.precision == SHT_MIXED) != mixed_groups || r != cudaSuccess) continue;
        const int4 *items = stage ? g.d_ana[polar] : g.d_syn[polar];
        const int ni = stage ? g.nana[polar] : g.nsyn[polar];
        if (stage == 0 && g.tc)
          r = launch_leg_tc_batch(g.spin, g.nj, g.d_targs[polar], items, ni, s);
        else if (stage == 1 && g.tca)
          r = launch_leg_tc_ana_batch(g.spin, g.nj, g.d_targs[polar], items, ni, s);
        else
          r = mixed_groups ? launch_leg_mixed_batch(stage, g.spin, g.nj, g.ppt, g.d_args[polar], items, ni, TA, s)
                           : launch_leg_fp64_batch(stage, g.spin, g.nj, g.ppt, g.d_args[polar], items, ni, TA, s);
      }
      return r;
    };
    if (has[0] && has[1])
      return fork_join(
          st, B->side, B->ev_fork, B->ev_join, [&](cudaStream_t s) { return run(true, s); },
          [&](cudaStream_t s) { return run(false, s); });
    return run(has[1], st);
  };
  if (type == SHT_SYNTHESIS || type == SHT_ADJOINT_ANALYSIS) {
    const int weighted = type == SHT_ADJOINT_ANALYSIS;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
      const sht_plan_s *P = B->plans[k];
      e = P->precision == SHT_MIXED ? launch_alm_prepare_mixed(P, A[k], st) : launch_alm_prepare_fp64(P, A[k], st);
      if (e == cudaSuccess && P->precision == SHT_MIXED && P->nsyn_lo[polar])  // its FP64 columns
        e = launch_alm_prepare_fp64(P, A[k], st);
    }
    if (e == cudaSuccess) e = legendre(0);
    for (int df = 0; df < 2 && e == cudaSuccess; ++df)
      e = launch_fft_batch(0, df, B->d_fft_syn[polar][weighted][add], B->d_fft_items[df], B->nfft_items[df],
                           B->fft_smem, TM, st);
  } else {
    const int weighted = type == SHT_ANALYSIS;
    for (int df = 0; df < 2 && e == cudaSuccess; ++df)
      e = launch_fft_batch(1, df, B->d_fft_ana[weighted], B->d_fft_items[df], B->nfft_items[df], B->fft_smem, TM, st);
    if (e == cudaSuccess) e = legendre(1);
    for (int k = 0; k < n && e == cudaSuccess; ++k) e = launch_ana_reduce(B->plans[k], A[k], polar, add, st);
  }
  if (cur != B->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return SHT_OK;
}
