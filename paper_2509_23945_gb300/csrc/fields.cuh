// Held-layer field energies of an active slice site (shared by the tensor-network
// and the learned proposals).
#pragma once

#include "common.cuh"

namespace tnmc {

// Integer field energies h(v) = sum over bonds of (r, x) not carried by the
// slice network of J * e(v, neighbour): held layers, fixed line / column and
// the zero-valued wraps of open axes.
__device__ inline void site_field(const Group& g, const SliceGeom& s, const int8_t* spins, const int32_t* J,
                                  int r, int x, long long* h) {
  const int d = g.d;
  for (int v = 0; v < d; ++v) h[v] = 0;
  const int idx = site_index(g, s, r, x);
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  for (int a = 0; a < 3; ++a) {
    bool out_carried = false, in_carried = false;
    if (a == s.ca) { out_carried = (x + 1 < s.Lc) || s.ring; in_carried = (x >= 1) || s.ring; }
    if (a == s.ra) { out_carried = (r < s.m); in_carried = (r >= 2); }
    if (!out_carried) {
      const int nb = shift_index(g, idx, a, +1);
      const long long j = J[a * vol + idx];
      const int sv = spins[nb];
      for (int v = 0; v < d; ++v) h[v] += j * pair_e(g.model, v, sv);
    }
    if (!in_carried) {
      const int nb = shift_index(g, idx, a, -1);
      const long long j = J[a * vol + nb];
      const int sv = spins[nb];
      for (int v = 0; v < d; ++v) h[v] += j * pair_e(g.model, v, sv);
    }
  }
}

}  // namespace tnmc
