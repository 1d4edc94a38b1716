// Single-spin Metropolis on the context's lattices: the paper's comparison
// method (main text, "Sampling 3D spin glasses"; SM III first-passage times).
//
// A spin s_i (Ising value 1 - 2 index) flips with probability
// min(1, exp(-beta dE)), dE = 2 s_i h_i, h_i = sum_j J_ij s_j, in two
// checkerboard half-sweeps per sweep (colour (x + y + z) mod 2). Sites of one
// colour share no bond on a bipartite lattice (open axes or even periodic
// extents), so one thread per site updates a half-sweep in place. The uniform
// of site i in half-sweep c of sweep t is Philox purpose 7, index i, slice c,
// axis 0, step t, global chain id.
#include <vector>

#include "../../include/tnmc.h"
#include "common.cuh"

using namespace tnmc;

namespace {

constexpr uint32_t kPurposeMetro = 7;

__global__ void metropolis_half_sweep(Group g, uint64_t seed, uint32_t t, int colour, unsigned int* acc) {
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  const size_t total = vol * (size_t)g.n_chains;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int chain = (int)(e / vol);
    const int i = (int)(e - (size_t)chain * vol);
    const int x = i % g.L[0], y = (i / g.L[0]) % g.L[1], z = i / (g.L[0] * g.L[1]);
    if (((x + y + z) & 1) != colour) continue;
    int8_t* s = g.spins + (size_t)chain * vol;
    const int32_t* J = g.J + (size_t)g.inst[chain] * 3 * vol;
    long long h = 0;
    for (int a = 0; a < 3; ++a) {
      const int up = shift_index(g, i, a, +1), dn = shift_index(g, i, a, -1);
      h += (long long)J[a * vol + i] * (1 - 2 * s[up]) + (long long)J[a * vol + dn] * (1 - 2 * s[dn]);
    }
    const int si = 1 - 2 * s[i];
    const long long dE = 2LL * si * h;
    const double u = philox_uniform(seed, kPurposeMetro, (uint32_t)i, (uint32_t)colour, 0, t,
                                    (uint32_t)(g.chain_base + chain));
    const double beta = g.beta[chain];
    if (u < exp(fmin(0.0, -beta * (double)dE * kJScale))) {
      s[i] = (int8_t)(1 - s[i]);
      if (acc) atomicAdd(acc + g.chain_base + chain, 1u);
    }
  }
}

}  // namespace

// Entry point used by tnmc_api.cu (which owns the context): one half-sweep of one group.
void tnmc_launch_metropolis(const Group& g, uint64_t seed, uint32_t t, int colour, unsigned int* acc,
                            cudaStream_t stream) {
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  const size_t total = vol * (size_t)g.n_chains;
  const int threads = 256;
  size_t blocks = (total + threads - 1) / threads;
  if (blocks > 65535) blocks = 65535;
  metropolis_half_sweep<<<(unsigned)blocks, threads, 0, stream>>>(g, seed, t, colour, acc);
}
