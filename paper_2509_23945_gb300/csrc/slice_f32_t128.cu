// slice_update_kernel<float> with 128 x 64 CUDA-core GEMM tiles (same results as the default tile; the
// tuning's gemm_tile = 2 launches it) and its host entry points.
#define TNMC_GEMM_TILE 2
#include "slice_launch.cuh"

namespace tnmc {

cudaError_t slice_launch_f32_t128(const PhaseParams& P, int total_items, int grid, size_t dyn_bytes,
                                  cudaStream_t stream) {
  slice_update_kernel_t128<float><<<grid, kThreads, dyn_bytes, stream>>>(P, total_items);
  return cudaPeekAtLastError();
}

cudaError_t slice_attributes_f32_t128(cudaFuncAttributes* fa) {
  return cudaFuncGetAttributes(fa, slice_update_kernel_t128<float>);
}

cudaError_t slice_set_dyn_smem_f32_t128(int bytes) {
  return cudaFuncSetAttribute(slice_update_kernel_t128<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t slice_occupancy_f32_t128(int* ctas_per_sm, size_t dyn_bytes) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, slice_update_kernel_t128<float>, kThreads,
                                                       dyn_bytes);
}

}  // namespace tnmc
