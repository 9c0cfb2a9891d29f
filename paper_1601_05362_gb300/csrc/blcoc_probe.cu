// blcoc_probe_peak: measured FMA throughput of the current GPU (FP64 DFMA or FP32 FFMA),
// the denominator of the ALU roofline the row passes are reported against.
//
// The paper has no counterpart: it is a measuring utility.  Every thread runs eight
// independent FMA chains (x <- x a + b, |a| < 1, so the values stay bounded) for a fixed
// number of steps; one wave of CTAs fills every SM to its thread limit, so the FMA pipe,
// not the dependency latency, bounds the kernel.  The result is stored only under a
// condition the values never meet, which keeps the chains live without memory traffic.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/blcoc.h"
#include "blcoc_common.cuh"

namespace blcoc {

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(T* out, int steps, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)c;
  for (int i = 0; i < steps; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = x[0];
#pragma unroll
  for (int c = 1; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == (T)-1) out[0] = s;   // never true: the chains stay positive
}

template <typename T>
blcoc_status run_probe(int steps, double* flops_per_s) {
  char msg[200];
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, PROBE_THREADS, 0);
  T* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(T));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  float best = 0.f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {   // one warm-up launch, best of three
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      k_fma_probe<T><<<grid, PROBE_THREADS, 0, s>>>(out, steps, (T)0.999999, (T)1e-6);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  if (e != cudaSuccess || best <= 0.f) {
    snprintf(msg, sizeof msg, "blcoc_probe_peak: %s", e != cudaSuccess ? cudaGetErrorString(e) : "no timing");
    set_global_error(msg);
    return e == cudaErrorMemoryAllocation ? BLCOC_ERR_OOM : BLCOC_ERR_CUDA;
  }
  const double flops = 2.0 * PROBE_CHAINS * (double)steps * (double)grid * PROBE_THREADS;
  *flops_per_s = flops / (best * 1e-3);
  return BLCOC_OK;
}

}  // namespace

}  // namespace blcoc

extern "C" blcoc_status blcoc_probe_peak(int kind, double* flops_per_s) {
  if (!flops_per_s || (kind != 0 && kind != 1)) {
    blcoc::set_global_error("blcoc_probe_peak: kind must be 0 (FP64) or 1 (FP32) and flops_per_s non-NULL");
    return BLCOC_ERR_INVALID_ARG;
  }
  // about 0.05 s per launch on a GB300 at either precision
  return kind == 0 ? blcoc::run_probe<double>(16000, flops_per_s) : blcoc::run_probe<float>(1000000, flops_per_s);
}
