// Host entry points of slice_update_kernel<R>. The float and double instances are compiled in their
// own translation units (slice_f32.cu, slice_f64.cu), so the library's sources build in parallel and
// each instance is compiled once.
#pragma once

#include <cuda_runtime.h>

#include "slice_kernel.cuh"

namespace tnmc {

template <typename R>
cudaError_t slice_launch(const PhaseParams& P, int total_items, int grid, size_t dyn_bytes, cudaStream_t stream);
template <typename R>
cudaError_t slice_attributes(cudaFuncAttributes* fa);
template <typename R>
cudaError_t slice_set_dyn_smem(int bytes);
template <typename R>
cudaError_t slice_occupancy(int* ctas_per_sm, size_t dyn_bytes);

template <> cudaError_t slice_launch<float>(const PhaseParams&, int, int, size_t, cudaStream_t);
template <> cudaError_t slice_launch<double>(const PhaseParams&, int, int, size_t, cudaStream_t);
template <> cudaError_t slice_attributes<float>(cudaFuncAttributes*);
template <> cudaError_t slice_attributes<double>(cudaFuncAttributes*);
template <> cudaError_t slice_set_dyn_smem<float>(int);
template <> cudaError_t slice_set_dyn_smem<double>(int);
template <> cudaError_t slice_occupancy<float>(int*, size_t);
template <> cudaError_t slice_occupancy<double>(int*, size_t);

#ifdef TNMC_PROFILE
// Profiling builds: each translation unit holds its own tnmc_prof counters; read and reset them.
template <typename R>
void slice_prof_read(unsigned long long* out16);
template <> void slice_prof_read<float>(unsigned long long*);
template <> void slice_prof_read<double>(unsigned long long*);
#endif

}  // namespace tnmc
