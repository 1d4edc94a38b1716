// Host entry points of slice_update_kernel<R>. The float and double instances are compiled in their
// own translation units (slice_f32.cu, slice_f64.cu), so the library's sources build in parallel and
// each instance is compiled once.
#pragma once

#include <cuda_runtime.h>

#include "slice_kernel.cuh"

namespace tnmc {

// The float kernel is also compiled with 32 x 32 (tile 1, slice_f32_t32.cu) and 128 x 64 (tile 2,
// slice_f32_t128.cu) CUDA-core GEMM tiles and, as its own instance, with the tcgen05 GEMM engine
// (slice_f32_umma.cu). slice_launch<float> runs the tcgen05 instance for the UMMA engines, else the
// instance of P.gemm_tile; the attribute calls take the instance: 0, 1, 2 the tiles, 3 tcgen05. The
// double kernel has the default instance only.
template <typename R>
cudaError_t slice_launch(const PhaseParams& P, int total_items, int grid, size_t dyn_bytes, cudaStream_t stream);
template <typename R>
cudaError_t slice_attributes(cudaFuncAttributes* fa, int tile = 0);
template <typename R>
cudaError_t slice_set_dyn_smem(int bytes, int tile = 0);
template <typename R>
cudaError_t slice_occupancy(int* ctas_per_sm, size_t dyn_bytes, int tile = 0);

template <> cudaError_t slice_launch<float>(const PhaseParams&, int, int, size_t, cudaStream_t);
template <> cudaError_t slice_launch<double>(const PhaseParams&, int, int, size_t, cudaStream_t);
template <> cudaError_t slice_attributes<float>(cudaFuncAttributes*, int);
template <> cudaError_t slice_attributes<double>(cudaFuncAttributes*, int);
template <> cudaError_t slice_set_dyn_smem<float>(int, int);
template <> cudaError_t slice_set_dyn_smem<double>(int, int);
template <> cudaError_t slice_occupancy<float>(int*, size_t, int);
template <> cudaError_t slice_occupancy<double>(int*, size_t, int);

// entry points of the float kernel's tile variants (tile 1: t32, tile 2: t128)
cudaError_t slice_launch_f32_t32(const PhaseParams&, int, int, size_t, cudaStream_t);
cudaError_t slice_attributes_f32_t32(cudaFuncAttributes*);
cudaError_t slice_set_dyn_smem_f32_t32(int);
cudaError_t slice_occupancy_f32_t32(int*, size_t);
cudaError_t slice_launch_f32_t128(const PhaseParams&, int, int, size_t, cudaStream_t);
cudaError_t slice_attributes_f32_t128(cudaFuncAttributes*);
cudaError_t slice_set_dyn_smem_f32_t128(int);
cudaError_t slice_occupancy_f32_t128(int*, size_t);
// the float kernel with the tcgen05 GEMM engine (instance 3)
constexpr int kSliceInstanceUmma = 3;
cudaError_t slice_launch_f32_umma(const PhaseParams&, int, int, size_t, cudaStream_t);
cudaError_t slice_attributes_f32_umma(cudaFuncAttributes*);
cudaError_t slice_set_dyn_smem_f32_umma(int);
cudaError_t slice_occupancy_f32_umma(int*, size_t);

#ifdef TNMC_PROFILE
// Profiling builds: each translation unit holds its own tnmc_prof counters; read and reset them.
template <typename R>
void slice_prof_read(unsigned long long* out16);
template <> void slice_prof_read<float>(unsigned long long*);
template <> void slice_prof_read<double>(unsigned long long*);
#endif

}  // namespace tnmc
