// Host-only stand-in for <cuda_runtime.h>, used by tests that compile the library's integer device
// helpers (slice geometry, composite-layer fields and bond tables, the sweep schedule) with a plain C++
// compiler to compare them with the oracle on a machine without CUDA devices. Qualifiers become empty
// and the thread index is a single thread.
#pragma once
#include <cmath>
#include <cstdint>
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
struct TnmcHostDim3 { unsigned x = 0, y = 0, z = 0; };
static TnmcHostDim3 threadIdx, blockIdx, blockDim, gridDim;
template <typename T> inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
inline void __syncthreads() {}
