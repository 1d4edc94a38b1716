// Held-layer field energies of an active slice site (shared by the tensor-network
// and the learned proposals).
#pragma once

#include "common.cuh"

namespace tnmc {

// ------------------------------------------------------------ TNMCMC-2 superspins
// A composite layer (SM II.B) joins layers k and k + 1 along the slice normal; the superspin at
// active site (r, x) has state v = a + 2 b with a, b the state indices of its layer-k and
// layer-(k + 1) spins.

// Lattice index of the spin of `layer` (0: k, 1: k + 1) under active site (r, x).
__device__ inline int layer_index(const Group& g, const SliceGeom& s, int r, int x, int layer) {
  const int idx = site_index(g, s, r, x);
  return layer ? shift_index(g, idx, s.axis, +1) : idx;
}

// Current state of active site (r, x): the spin, or the superspin of a composite layer.
__device__ inline int read_site(const Group& g, const SliceGeom& s, const int8_t* spins, int r, int x) {
  const int idx = site_index(g, s, r, x);
  if (g.layers != 2) return spins[idx];
  return spins[idx] + 2 * spins[shift_index(g, idx, s.axis, +1)];
}

__device__ inline void write_site(const Group& g, const SliceGeom& s, int8_t* spins, int r, int x, int v) {
  const int idx = site_index(g, s, r, x);
  if (g.layers != 2) { spins[idx] = (int8_t)v; return; }
  spins[idx] = (int8_t)(v & 1);
  spins[shift_index(g, idx, s.axis, +1)] = (int8_t)(v >> 1);
}

// Integer energy factor of the in-plane bond stored at active site (r, x) (lattice index idx) along
// axis ba, between states v at (r, x) and w at its neighbour: J e(v, w), or for superspins the sum
// over both layers J_k e(a, a') + J_k+1 e(b, b').
__device__ inline long long bond_energy(const Group& g, const SliceGeom& s, const int32_t* J, size_t vol, int idx,
                                        int ba, int v, int w) {
  if (g.layers != 2) return (long long)J[ba * vol + idx] * pair_e(g.model, v, w);
  const int idx1 = shift_index(g, idx, s.axis, +1);
  return (long long)J[ba * vol + idx] * pair_e(g.model, v & 1, w & 1) +
         (long long)J[ba * vol + idx1] * pair_e(g.model, v >> 1, w >> 1);
}

// Field energies h(v), v = 0..3, of the superspin at (r, x): the in-plane bonds the network does not
// carry (fixed line / column, zero-valued open wraps) of both layers, the held layers k - 1 and
// k + 2, and the bonds between the two spins. Each lattice bond record is counted once: the bond
// from layer k to layer k + 1 is taken from layer k; on an axis of extent 2 the wrapping bond from
// layer k + 1 back to layer k joins the same two spins and is taken from layer k as well.
__device__ inline void composite_field(const Group& g, const SliceGeom& s, const int8_t* spins, const int32_t* J,
                                       int r, int x, long long* h) {
  for (int v = 0; v < 4; ++v) h[v] = 0;
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  const int two = g.L[s.axis] == 2;
  for (int layer = 0; layer < 2; ++layer) {
    const int idx = layer_index(g, s, r, x, layer);
    for (int a = 0; a < 3; ++a) {
      if (a == s.axis) {
        const int nb_out = shift_index(g, idx, a, +1), nb_in = shift_index(g, idx, a, -1);
        const long long j_out = J[a * vol + idx], j_in = J[a * vol + nb_in];
        if (layer == 0) {
          // out: to layer k + 1 (internal); in: from layer k - 1 (held), or from layer k + 1 on extent 2
          for (int v = 0; v < 4; ++v) h[v] += j_out * pair_e(g.model, v & 1, v >> 1);
          if (two) {
            for (int v = 0; v < 4; ++v) h[v] += j_in * pair_e(g.model, v & 1, v >> 1);
          } else {
            const int sv = spins[nb_in];
            for (int v = 0; v < 4; ++v) h[v] += j_in * pair_e(g.model, v & 1, sv);
          }
        } else if (!two) {
          // in: from layer k (internal, counted above); out: to layer k + 2 (held)
          const int sv = spins[nb_out];
          for (int v = 0; v < 4; ++v) h[v] += j_out * pair_e(g.model, v >> 1, sv);
        }
        continue;
      }
      bool out_carried = false, in_carried = false;
      if (a == s.ca) { out_carried = (x + 1 < s.Lc) || s.ring; in_carried = (x >= 1) || s.ring; }
      if (a == s.ra) { out_carried = (r < s.m); in_carried = (r >= 2); }
      if (!out_carried) {
        const int sv = spins[shift_index(g, idx, a, +1)];
        const long long j = J[a * vol + idx];
        for (int v = 0; v < 4; ++v) h[v] += j * pair_e(g.model, (v >> layer) & 1, sv);
      }
      if (!in_carried) {
        const int nb = shift_index(g, idx, a, -1);
        const long long j = J[a * vol + nb];
        const int sv = spins[nb];
        for (int v = 0; v < 4; ++v) h[v] += j * pair_e(g.model, (v >> layer) & 1, sv);
      }
    }
  }
}

// Integer field energies h(v) = sum over bonds of (r, x) not carried by the
// slice network of J * e(v, neighbour): held layers, fixed line / column and
// the zero-valued wraps of open axes.
__device__ inline void site_field(const Group& g, const SliceGeom& s, const int8_t* spins, const int32_t* J,
                                  int r, int x, long long* h) {
  if (g.layers == 2) {
    composite_field(g, s, spins, J, r, x, h);
    return;
  }
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
