// slice_update_kernel<float> and its host entry points.
#include "slice_launch.cuh"

namespace tnmc {

template <>
cudaError_t slice_launch<float>(const PhaseParams& P, int total_items, int grid, size_t dyn_bytes, cudaStream_t stream) {
  if (P.gemm_mode == GEMM_UMMA_TF32X3 || P.gemm_mode == GEMM_UMMA_BF16)
    return slice_launch_f32_umma(P, total_items, grid, dyn_bytes, stream);
  if (P.gemm_tile == 1) return slice_launch_f32_t32(P, total_items, grid, dyn_bytes, stream);
  if (P.gemm_tile == 2) return slice_launch_f32_t128(P, total_items, grid, dyn_bytes, stream);
  slice_update_kernel<float><<<grid, kThreads, dyn_bytes, stream>>>(P, total_items);
  return cudaPeekAtLastError();   // not cleared: the caller checks the launch
}

template <>
cudaError_t slice_attributes<float>(cudaFuncAttributes* fa, int tile) {
  if (tile == kSliceInstanceUmma) return slice_attributes_f32_umma(fa);
  if (tile == 1) return slice_attributes_f32_t32(fa);
  if (tile == 2) return slice_attributes_f32_t128(fa);
  return cudaFuncGetAttributes(fa, slice_update_kernel<float>);
}

template <>
cudaError_t slice_set_dyn_smem<float>(int bytes, int tile) {
  if (tile == kSliceInstanceUmma) return slice_set_dyn_smem_f32_umma(bytes);
  if (tile == 1) return slice_set_dyn_smem_f32_t32(bytes);
  if (tile == 2) return slice_set_dyn_smem_f32_t128(bytes);
  return cudaFuncSetAttribute(slice_update_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <>
cudaError_t slice_occupancy<float>(int* ctas_per_sm, size_t dyn_bytes, int tile) {
  if (tile == kSliceInstanceUmma) return slice_occupancy_f32_umma(ctas_per_sm, dyn_bytes);
  if (tile == 1) return slice_occupancy_f32_t32(ctas_per_sm, dyn_bytes);
  if (tile == 2) return slice_occupancy_f32_t128(ctas_per_sm, dyn_bytes);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, slice_update_kernel<float>, kThreads, dyn_bytes);
}

#ifdef TNMC_PROFILE
template <>
void slice_prof_read<float>(unsigned long long* out16) {
  cudaMemcpyFromSymbol(out16, tnmc_prof, sizeof(unsigned long long) * 16);
  unsigned long long z[16] = {0};
  cudaMemcpyToSymbol(tnmc_prof, z, sizeof(z));
}
#endif

}  // namespace tnmc
