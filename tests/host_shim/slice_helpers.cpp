// Prints the slice (argument "1") or composite-layer quantities of the library's device helpers for one lattice read from stdin,
// and the composite schedule for small extents (see tests/test_host_slice_helpers.py).
#include <cstdio>
#include <vector>
#include "fields.cuh"
using namespace tnmc;
int main(int argc, char** argv) {
  // argument "1": a TNMCMC-1 slice (site fields and bond energies of d-state spins); default: a composite layer
  const bool single = argc > 1 && argv[1][0] == '1';
  int L[3], bc[3], model, fix, axis, k;
  unsigned long long seed;
  unsigned step, chain;
  if (scanf("%d %d %d %d %d %d %d %d %d %d %llu %u %u", &L[0], &L[1], &L[2], &bc[0], &bc[1], &bc[2], &model, &fix,
            &axis, &k, &seed, &step, &chain) != 13)
    return 1;
  const int vol = L[0] * L[1] * L[2];
  std::vector<int8_t> spins(vol);
  std::vector<int32_t> J(3 * vol);
  for (int i = 0; i < vol; ++i) {
    int v;
    if (scanf("%d", &v) != 1) return 1;
    spins[i] = (int8_t)v;
  }
  for (int i = 0; i < 3 * vol; ++i)
    if (scanf("%d", &J[i]) != 1) return 1;
  Group g{};
  for (int a = 0; a < 3; ++a) { g.L[a] = L[a]; g.bc[a] = bc[a]; }
  g.model = model; g.d = 4; g.fix_mode = fix; g.layers = 2;
  if (single) { g.d = model == 2 ? 3 : 2; g.layers = 1; }
  const SliceGeom s = make_geom(g, axis, k, seed, step, chain);
  printf("%d %d %d %d\n", s.m, s.Lc, s.y0, s.x0);
  if (single) {
    const int d = g.d;
    for (int r = 1; r <= s.m; ++r)
      for (int x = 0; x < s.Lc; ++x) {
        long long h[4];
        site_field(g, s, spins.data(), J.data(), r, x, h);
        const int idx = site_index(g, s, r, x);
        printf("%d", read_site(g, s, spins.data(), r, x));
        for (int v = 0; v < d; ++v) printf(" %lld", h[v]);
        for (int kind = 0; kind < 2; ++kind) {
          const bool present = kind == 0 ? ((x + 1 < s.Lc) || s.ring) : (r < s.m);
          for (int v = 0; v < d; ++v)
            for (int u = 0; u < d; ++u)
              printf(" %lld", present ? bond_energy(g, s, J.data(), (size_t)vol, idx, kind == 0 ? s.ca : s.ra, v, u) : 0LL);
        }
        printf("\n");
      }
    return 0;
  }
  for (int r = 1; r <= s.m; ++r)
    for (int x = 0; x < s.Lc; ++x) {
      long long h[4];
      composite_field(g, s, spins.data(), J.data(), r, x, h);
      const int idx = site_index(g, s, r, x);
      printf("%d", read_site(g, s, spins.data(), r, x));
      for (int v = 0; v < 4; ++v) printf(" %lld", h[v]);
      for (int kind = 0; kind < 2; ++kind) {
        const bool present = kind == 0 ? ((x + 1 < s.Lc) || s.ring) : (r < s.m);
        for (int v = 0; v < 4; ++v)
          for (int u = 0; u < 4; ++u)
            printf(" %lld", present ? bond_energy(g, s, J.data(), (size_t)vol, idx, kind == 0 ? s.ca : s.ra, v, u) : 0LL);
      }
      printf("\n");
    }
  for (int n = 2; n <= 9; ++n)
    for (int per = 0; per < 2; ++per)
      for (int off = 0; off < 2; ++off)
        for (int c = 0; c < 3; ++c) {
          printf("S %d %d %d %d :", n, per, off, c);
          for (int j = 0; j < composite_count(n, per, off, c); ++j) printf(" %d", composite_slice(n, per, off, c, j));
          printf("\n");
        }
  return 0;
}
