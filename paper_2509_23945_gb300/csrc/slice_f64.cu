// slice_update_kernel<double> and its host entry points.
#include "slice_launch.cuh"

namespace tnmc {

template <>
cudaError_t slice_launch<double>(const PhaseParams& P, int total_items, int grid, size_t dyn_bytes, cudaStream_t stream) {
  slice_update_kernel<double><<<grid, kThreads, dyn_bytes, stream>>>(P, total_items);
  return cudaPeekAtLastError();   // not cleared: the caller checks the launch
}

template <>
cudaError_t slice_attributes<double>(cudaFuncAttributes* fa, int) {
  return cudaFuncGetAttributes(fa, slice_update_kernel<double>);
}

template <>
cudaError_t slice_set_dyn_smem<double>(int bytes, int) {
  return cudaFuncSetAttribute(slice_update_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <>
cudaError_t slice_occupancy<double>(int* ctas_per_sm, size_t dyn_bytes, int) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, slice_update_kernel<double>, kThreads, dyn_bytes);
}

#ifdef TNMC_PROFILE
template <>
void slice_prof_read<double>(unsigned long long* out16) {
  cudaMemcpyFromSymbol(out16, tnmc_prof, sizeof(unsigned long long) * 16);
  unsigned long long z[16] = {0};
  cudaMemcpyToSymbol(tnmc_prof, z, sizeof(z));
}
#endif

}  // namespace tnmc
