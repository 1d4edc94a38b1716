// tnmc_probe_alu_peak: measured FP32 / FP64 fused multiply-add throughput of the
// current device, the denominator of the slice kernel's roofline (the slice
// update is bound by CUDA-core arithmetic, not by HBM or the tensor cores).
//
// Every thread runs 8 independent FMA chains for a fixed number of iterations;
// the grid fills every SM with 8 CTAs of 256 threads, so the FMA pipes, not
// latency, set the rate. The launch is timed with CUDA events on the given
// stream after one untimed launch; flops = 2 x FMAs.
#include <cuda_runtime.h>

#include "../../include/tnmc.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;
constexpr int kChains = 8;

__device__ double g_probe_sink;   // keeps the chains live; written only if a result is impossible

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)-1.2345e30) g_probe_sink = (double)s;
}

template <typename T>
tnmc_status run_probe(cudaStream_t stream, int iters, double* out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TNMC_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TNMC_ERR_CUDA;
  const int grid = sms * kProbeCtasPerSm;
  // b < 1 and c small keep the chains finite for any iteration count
  const T b = (T)0.999, c = (T)1e-3;
  fma_probe_kernel<T><<<grid, kProbeThreads, 0, stream>>>(iters / 8 > 0 ? iters / 8 : 1, b, c);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TNMC_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return TNMC_ERR_CUDA; }
  cudaEventRecord(e0, stream);
  fma_probe_kernel<T><<<grid, kProbeThreads, 0, stream>>>(iters, b, c);
  cudaEventRecord(e1, stream);
  tnmc_status st = TNMC_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || !(ms > 0.f))
    st = TNMC_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TNMC_OK) return st;
  const double fmas = (double)grid * kProbeThreads * (double)iters * 16.0 * kChains;
  *out = 2.0 * fmas / (ms * 1e-3);
  return TNMC_OK;
}

}  // namespace

extern "C" tnmc_status tnmc_probe_alu_peak(int precision, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s) return TNMC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (precision == TNMC_PREC_F32) return run_probe<float>(s, 4096, flops_per_s);
  if (precision == TNMC_PREC_F64) return run_probe<double>(s, 256, flops_per_s);
  return TNMC_ERR_ARG;
}
