// FMA-throughput probe: the measured denominators of the forward kernels'
// rooflines.  The forward scatter is bound by FP32 (mixed form) or FP64
// (plain form) fused multiply-add issue, not by a dense contraction, so its
// roof is the rate at which the SMs retire independent FMA chains.
//
// Every thread runs kChains independent chains x <- x * b + c for `iters`
// rounds (b just below 1, so the chains stay bounded and never denormal);
// enough warps are resident that the FMA pipes, not latency, bound the rate.
// Work per launch: 2 x kChains x iters flop per thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/fwh.h"
#include "fwh_internal.cuh"

fwh_status fwh_fail_handle(fwh_handle h, fwh_status st, const char *msg);

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T b, T c, int iters, T *sink) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
  }
  T s = x[0];
#pragma unroll
  for (int i = 1; i < kChains; ++i) s += x[i];
  if (s == (T)-1) *sink = s;  // never true (every chain stays positive); keeps the work
}

template <typename T>
fwh_status run(int iters, double *tflops, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0);
  T *sink = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(T));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * std::max(1, std::min(per_sm, 4));
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>((T)0.999, (T)1e-3, iters / 8, sink);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>((T)0.999, (T)1e-3, iters, sink);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess)
    return fwh_fail_handle(nullptr, FWH_ERR_CUDA,
                           (std::string("fwh_fma_peak: ") + cudaGetErrorString(e)).c_str());
  const double flop = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flop / (ms * 1e-3) / 1e12;
  return FWH_OK;
}

}  // namespace

extern "C" fwh_status fwh_fma_peak(int precision, double *tflops, void *stream) {
  if (!tflops) return fwh_fail_handle(nullptr, FWH_ERR_ARG, "tflops is NULL");
  if (precision != FWH_FP64 && precision != FWH_MIXED)
    return fwh_fail_handle(nullptr, FWH_ERR_ARG, "precision must be FWH_FP64 or FWH_MIXED");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // about 60 ms per timed launch on a GB300 for either precision
  return precision == FWH_FP64 ? run<double>(1 << 15, tflops, s) : run<float>(1 << 21, tflops, s);
}
