// slice_update_kernel<float> with the tcgen05 GEMM engine compiled in (gemm_mode UMMA_TF32X3 or
// UMMA_BF16 launches it) and its host entry points. The other instances carry no tensor-memory code.
#define TNMC_WITH_UMMA 1
#include "slice_launch.cuh"

namespace tnmc {

cudaError_t slice_launch_f32_umma(const PhaseParams& P, int total_items, int grid, size_t dyn_bytes,
                                  cudaStream_t stream) {
  slice_update_kernel_umma<float><<<grid, kThreads, dyn_bytes, stream>>>(P, total_items);
  return cudaPeekAtLastError();
}

cudaError_t slice_attributes_f32_umma(cudaFuncAttributes* fa) {
  return cudaFuncGetAttributes(fa, slice_update_kernel_umma<float>);
}

cudaError_t slice_set_dyn_smem_f32_umma(int bytes) {
  return cudaFuncSetAttribute(slice_update_kernel_umma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t slice_occupancy_f32_umma(int* ctas_per_sm, size_t dyn_bytes) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, slice_update_kernel_umma<float>, kThreads,
                                                       dyn_bytes);
}

}  // namespace tnmc
