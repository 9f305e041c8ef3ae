// peaks.cu -- throughput of the arithmetic pipes the transforms run on, measured
// on the device at hand (the denominators of the kernels' rooflines: the FP64
// form is bound by the FP64 pipe, the mixed form by FP32 issue).
//
// Every thread runs kChains independent chains (x = x b + c, or x = x + c) for a
// given number of steps, so that issue rather than latency limits the rate; the
// grid holds 8 CTAs of 256 threads per SM.  Each thread writes its sum, so no
// chain can be dropped.
#include <algorithm>

#include "sht_internal.h"

namespace sht {

constexpr int kPeakChains = 8, kPeakThreads = 256, kPeakCtasPerSm = 8;

template <class T, bool FMA>
__global__ void __launch_bounds__(kPeakThreads) pipe_kernel(T *out, int iters, T b, T c) {
  T x[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < iters; it += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < kPeakChains; ++i) {
        if constexpr (sizeof(T) == 8) {
          x[i] = FMA ? __fma_rn(x[i], b, c) : __dadd_rn(x[i], c);
        } else {
          x[i] = FMA ? __fmaf_rn(x[i], b, c) : __fadd_rn(x[i], c);
        }
      }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// operations per second of one kernel: one untimed launch, then the best of three
template <class T, bool FMA>
static cudaError_t time_pipe(int nsm, int iters, T *buf, cudaStream_t st, double *ops_per_s) {
  const int grid = nsm * kPeakCtasPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      pipe_kernel<T, FMA><<<grid, kPeakThreads, 0, st>>>(buf, iters, (T)0.999999, (T)1e-6);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess)
    *ops_per_s = (double)grid * kPeakThreads * kPeakChains * (double)iters / (best * 1e-3);
  return e;
}

}  // namespace sht

using namespace sht;

extern "C" int sht_measure_pipe_peaks(int device, double *out) {
  if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
  int cur = -1, nsm = 0, ndev = 0;
  cudaGetDevice(&cur);
  if (device < 0) device = cur;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();  // leave no error behind for the caller's next launch check
    return set_error(SHT_ERR_INVALID_ARG, "device %d of %d", device, ndev);
  }
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t st = nullptr;
  void *buf = nullptr;
  const size_t n = (size_t)std::max(nsm, 1) * kPeakCtasPerSm * kPeakThreads;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&buf, n * sizeof(double));
  double r[3] = {0, 0, 0};
  if (e == cudaSuccess) e = time_pipe<double, true>(nsm, 2048, (double *)buf, st, &r[0]);
  if (e == cudaSuccess) e = time_pipe<float, true>(nsm, 65536, (float *)buf, st, &r[1]);
  if (e == cudaSuccess) e = time_pipe<float, false>(nsm, 65536, (float *)buf, st, &r[2]);
  if (buf) cudaFree(buf);
  if (st) cudaStreamDestroy(st);
  if (cur >= 0 && cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) return set_error(SHT_ERR_CUDA, "pipe measurement: %s", cudaGetErrorString(e));
  out[0] = 2.0 * r[0] * 1e-12;  // FP64 FMA: TFLOP/s, an FMA counted as 2 flops
  out[1] = r[1] * 1e-12;        // FP32 FMA: T op/s
  out[2] = r[2] * 1e-12;        // FP32 add: T op/s
  return SHT_OK;
}
