// tnmc_cta_gemm: the CTA-level GEMM engines of the slice kernel run on their own, one CTA per
// matrix of a batch, so each engine can be checked against a host product and timed at full
// occupancy outside the slice update.
#include <cuda_runtime.h>

#include "../../include/tnmc.h"
#include "linalg.cuh"
#include "tc_gemm.cuh"
#include "umma.cuh"

namespace {

using namespace tnmc;

__device__ unsigned int g_gemm_status;

struct GemmArgs {
  int M, N, K, lda, ldb, ldc, ta, tb;
  float alpha, beta;
  const float* A;
  const float* B;
  float* C;
  long long sA, sB, sC;
};

template <int ENGINE>
__global__ void __launch_bounds__(kThreads) cta_gemm_kernel(GemmArgs g) {
  const float* A = g.A + (size_t)blockIdx.x * g.sA;
  const float* B = g.B + (size_t)blockIdx.x * g.sB;
  float* C = g.C + (size_t)blockIdx.x * g.sC;
  if constexpr (ENGINE == TNMC_GEMM_FFMA) {
    __shared__ GemmSmem<float> sm;
    cta_gemm<float>(g.M, g.N, g.K, g.alpha, A, g.lda, g.ta, B, g.ldb, g.tb, g.beta, C, g.ldc, sm);
  } else if constexpr (ENGINE == TNMC_GEMM_MMA_TF32X3 || ENGINE == TNMC_GEMM_MMA_BF16) {
    __shared__ TcGemmSmem sm;
    cta_gemm_tc(ENGINE == TNMC_GEMM_MMA_BF16 ? GEMM_BF16 : GEMM_TF32X3, g.M, g.N, g.K, g.alpha, A, g.lda, g.ta, B,
                g.ldb, g.tb, g.beta, C, g.ldc, sm);
  } else {
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ UmmaCtl ctl;
    cta_gemm_umma<ENGINE == TNMC_GEMM_UMMA_BF16 ? UMMA_BF16 : UMMA_TF32X3>(
        g.M, g.N, g.K, g.alpha, A, g.lda, g.ta, B, g.ldb, g.tb, g.beta, C, g.ldc, dyn, ctl, &g_gemm_status);
  }
}

template <int ENGINE>
cudaError_t launch(const GemmArgs& g, int batch, cudaStream_t s) {
  size_t dyn = 0;
  if (ENGINE == TNMC_GEMM_UMMA_TF32X3 || ENGINE == TNMC_GEMM_UMMA_BF16) {
    dyn = kUmmaStageBytes;
    cudaError_t e = cudaFuncSetAttribute(cta_gemm_kernel<ENGINE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  cta_gemm_kernel<ENGINE><<<batch, kThreads, dyn, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

extern "C" tnmc_status tnmc_cta_gemm(int engine, int batch, int M, int N, int K, float alpha, const float* A, int lda,
                                     long long strideA, int transA, const float* B, int ldb, long long strideB,
                                     int transB, float beta, float* C, int ldc, long long strideC,
                                     void* cuda_stream) {
  if (engine < TNMC_GEMM_FFMA || engine > TNMC_GEMM_UMMA_BF16 || batch < 0 || batch > 65535 || M < 0 || N < 0 ||
      K < 0 || lda < 1 || ldb < 1 || ldc < 1 || strideA < 0 || strideB < 0 || strideC < 0)
    return TNMC_ERR_ARG;
  if (batch == 0 || M == 0 || N == 0) return TNMC_OK;
  if (!C || (K > 0 && (!A || !B))) return TNMC_ERR_ARG;
  if ((K > 0 && ((transA ? lda < M : lda < K) || (transB ? ldb < K : ldb < N))) || ldc < N) return TNMC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const unsigned int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_gemm_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TNMC_ERR_CUDA;
  GemmArgs g{M, N, K, lda, ldb, ldc, transA ? 1 : 0, transB ? 1 : 0, alpha, beta, A, B, C, strideA, strideB, strideC};
  cudaError_t e;
  switch (engine) {
    case TNMC_GEMM_FFMA: e = launch<TNMC_GEMM_FFMA>(g, batch, s); break;
    case TNMC_GEMM_MMA_TF32X3: e = launch<TNMC_GEMM_MMA_TF32X3>(g, batch, s); break;
    case TNMC_GEMM_MMA_BF16: e = launch<TNMC_GEMM_MMA_BF16>(g, batch, s); break;
    case TNMC_GEMM_UMMA_TF32X3: e = launch<TNMC_GEMM_UMMA_TF32X3>(g, batch, s); break;
    default: e = launch<TNMC_GEMM_UMMA_BF16>(g, batch, s); break;
  }
  if (e != cudaSuccess) return TNMC_ERR_CUDA;
  unsigned int st = 0;
  if (cudaMemcpyFromSymbolAsync(&st, g_gemm_status, sizeof(st), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TNMC_ERR_CUDA;
  return (st & ST_TIMEOUT) ? TNMC_ERR_TIMEOUT : TNMC_OK;
}
