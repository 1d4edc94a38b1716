// Shared device definitions of the slice-update library: Philox draws,
// lattice/group descriptors and small CTA helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Optional per-phase cycle counters (compile with -DTNMC_PROFILE): thread 0 of
// each CTA adds clock64() deltas to tnmc_prof[phase]. Off by default.
#ifdef TNMC_PROFILE
__device__ unsigned long long tnmc_prof[16];
#define TNMC_PROF_BEGIN(k) long long _pb##k = clock64()
#define TNMC_PROF_END(k) \
  if (threadIdx.x == 0) atomicAdd(&tnmc_prof[k], (unsigned long long)(clock64() - _pb##k))
#else
#define TNMC_PROF_BEGIN(k)
#define TNMC_PROF_END(k)
#endif

namespace tnmc {

constexpr int kThreads = 256;          // threads per CTA of the slice kernels
constexpr int kWarps = kThreads / 32;
constexpr int kJFracBits = 20;         // couplings are int32 in units of 2^-20
constexpr double kJScale = 1.0 / 1048576.0;
constexpr double kFloorEps = 1e-12;    // floor of truncated conditionals (eps * sum)

// Philox purposes. Proposal 0 of an environment build draws with P_SITE / P_MH; proposals j >= 1 of
// the same build with P_SITE_K (index (j - 1) * active sites + site) and P_MH_K (index j - 1).
enum Purpose : uint32_t { P_SITE = 0, P_FIXED_ROW = 1, P_FIXED_COL = 2, P_MH = 3, P_NET_SITE = 4, P_SITE_K = 5,
                          P_MH_K = 6 };

// Bits of the device status word a kernel latches for the next synchronising call.
enum StatusBits : int { ST_NONFINITE = 1, ST_TIMEOUT = 2 };

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
// multiplies with the published round constants; the key is bumped by the
// Weyl constants between rounds.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c[0];
    const uint64_t p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// Uniform double in [0, 1) from the top 53 bits of (o0 << 32 | o1).
__host__ __device__ inline double philox_uniform(uint64_t seed, uint32_t purpose, uint32_t index,
                                                 uint32_t slice, uint32_t axis, uint32_t step,
                                                 uint32_t chain) {
  uint32_t c[4] = {(purpose << 24) | index, slice | (axis << 16), step, chain};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t bits = ((uint64_t)c[0] << 32) | c[1];
  return (double)(bits >> 11) * (1.0 / 9007199254740992.0);
}

// One lattice geometry and its chains (device copy of tnmc_config + buffers).
struct Group {
  int L[3];
  int bc[3];
  int model;        // 0 EA +/-J, 1 EA Gaussian, 2 Potts
  int d;            // local states
  int chi;
  int fix_mode;     // 0 R1, 1 R2
  int n_chains;
  int chain_base;   // global chain id of chain 0 (Philox counter word)
  int8_t* spins;          // [n_chains][Lz][Ly][Lx]
  const int32_t* J;       // [n_inst][3][Lz][Ly][Lx]
  const double* beta;     // [n_chains]
  const int32_t* inst;    // [n_chains]
  int layers;             // 2: TNMCMC-2 composite layers of Ising superspins (d = 4); else TNMCMC-1
};

__host__ __device__ inline int pair_e(int model, int v, int w) {
  return model == 2 ? (v == w ? 1 : 0) : (1 - 2 * v) * (1 - 2 * w);
}

// Slices of one colour class along an axis of extent n: colours 0/1 are the
// even/odd slices; an odd periodic axis moves its last slice to colour 2.
__host__ __device__ inline int colour_count(int n, int periodic, int colour) {
  const bool three = periodic && (n % 2 == 1) && n > 1;
  const int top = three ? n - 1 : n;
  if (colour == 2) return three ? 1 : 0;
  return colour == 0 ? (top + 1) / 2 : top / 2;
}
__host__ __device__ inline int colour_slice(int n, int periodic, int colour, int j) {
  if (colour == 2) return n - 1;
  return 2 * j + colour;
}

// TNMCMC-2 schedule (SM II.B with the main text's pairs of contiguous layers): sweep t uses
// composite offset o = (t / 3) mod 2 and composites starting at layers o, o + 2, ... (both layers
// inside the lattice on an open axis). Composites j and j + 1 reach into each other's blanket, so
// they are coloured like TNMCMC-1 slices: a ring on a periodic axis of even extent, else a path.
__host__ __device__ inline int composite_total(int n, int periodic, int offset) {
  return periodic ? n / 2 : (n - offset) / 2;
}
__host__ __device__ inline int composite_count(int n, int periodic, int offset, int colour) {
  const int nc = composite_total(n, periodic, offset);
  return nc > 0 ? colour_count(nc, periodic && (n % 2 == 0), colour) : 0;
}
__host__ __device__ inline int composite_slice(int n, int periodic, int offset, int colour, int j) {
  const int nc = composite_total(n, periodic, offset);
  return (offset + 2 * colour_slice(nc, periodic && (n % 2 == 0), colour, j)) % n;
}

// Geometry of one slice update, as drawn for (seed, step). rax is the Philox axis word of every
// draw of the update: the axis, with bit 4 set for TNMCMC-2 composite layers.
struct SliceGeom {
  int axis, k, ra, ca, n_r, n_c, m, Lc, ring, row0, col0, y0, x0, rax;
};

// Geometry with given fixed row y0 and column x0 (-1: none; used only where the axis is periodic and,
// for x0, the fix mode is R2).
__device__ __host__ inline SliceGeom geom_with_lines(const Group& g, int axis, int k, int y0, int x0) {
  SliceGeom s;
  s.axis = axis; s.k = k;
  s.rax = axis | (g.layers == 2 ? 16 : 0);
  s.ca = (axis + 1) % 3; s.ra = (axis + 2) % 3;
  s.n_r = g.L[s.ra]; s.n_c = g.L[s.ca];
  if (g.bc[s.ra]) {
    s.y0 = y0; s.m = s.n_r - 1; s.row0 = y0;
  } else {
    s.y0 = -1; s.m = s.n_r; s.row0 = -1;
  }
  if (g.bc[s.ca] && g.fix_mode == 1) {
    s.x0 = x0; s.Lc = s.n_c - 1; s.col0 = x0 + 1; s.ring = 0;
  } else {
    s.x0 = -1; s.Lc = s.n_c; s.col0 = 0; s.ring = g.bc[s.ca] ? 1 : 0;
  }
  return s;
}

// Geometry of the update of (axis, k) at (seed, step): the fixed row / column are Philox draws.
__device__ __host__ inline SliceGeom make_geom(const Group& g, int axis, int k, uint64_t seed,
                                               uint32_t step, uint32_t gchain) {
  const uint32_t rax = axis | (g.layers == 2 ? 16 : 0);
  const int ra = (axis + 2) % 3, ca = (axis + 1) % 3;
  int y0 = -1, x0 = -1;
  if (g.bc[ra]) {
    const double u = philox_uniform(seed, P_FIXED_ROW, 0, k, rax, step, gchain);
    y0 = (int)(u * (double)g.L[ra]);
    if (y0 > g.L[ra] - 1) y0 = g.L[ra] - 1;
  }
  if (g.bc[ca] && g.fix_mode == 1) {
    const double u = philox_uniform(seed, P_FIXED_COL, 0, k, rax, step, gchain);
    x0 = (int)(u * (double)g.L[ca]);
    if (x0 > g.L[ca] - 1) x0 = g.L[ca] - 1;
  }
  return geom_with_lines(g, axis, k, y0, x0);
}

// Linear lattice index of active site (r in 1..m, x in 0..Lc-1).
__device__ __host__ inline int site_index(const Group& g, const SliceGeom& s, int r, int x) {
  int c[3];
  c[s.axis] = s.k;
  c[s.ra] = ((s.row0 + r) % s.n_r + s.n_r) % s.n_r;
  c[s.ca] = (s.col0 + x) % s.n_c;
  return (c[2] * g.L[1] + c[1]) * g.L[0] + c[0];
}

__device__ __host__ inline int shift_index(const Group& g, int idx, int a, int delta) {
  int c[3] = {idx % g.L[0], (idx / g.L[0]) % g.L[1], idx / (g.L[0] * g.L[1])};
  c[a] = (c[a] + delta + g.L[a]) % g.L[a];
  return (c[2] * g.L[1] + c[1]) * g.L[0] + c[0];
}

// ---------------------------------------------------------------- CTA helpers
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ inline T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Block-wide sum / max (all threads must call; result broadcast to all).
template <typename T>
__device__ inline T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kWarps ? red[threadIdx.x] : T(0);
    t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}
template <typename T>
__device__ inline T block_max(T v, T* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    T t = threadIdx.x < kWarps ? red[threadIdx.x] : red[0];
    t = warp_max(t);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  T t = red[0];
  __syncthreads();
  return t;
}

}  // namespace tnmc
