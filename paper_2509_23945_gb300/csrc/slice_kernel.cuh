// The fused TNMCMC-1 slice update: one CTA per (chain, slice) work item.
//
//   a1  held-layer fields and Boltzmann factors of the slice (SM II.A)
//   a2  boundary-MPS environments E_m = 1, E_{r-1} = trunc_chi(psiv * rowweight_r * E_r)
//       (SM I.B), truncation as below
//   a3  raster-order sampling of the candidate from the conditionals (SM I.C, Alg. 2)
//   a4  the same conditionals forced to the current slice: log q(current)
//   a5  exact integer energy difference and the acceptance of Eq. (1)
//
// Truncation (default route, the canonical SVD cut of SM I.B). The applied MPS
// B (bond n = chi * channels) is brought to right-canonical form from the right:
// M_x = B_x L_{x+1} (rows: left bond of x; columns: physical index and the
// columns of L_{x+1}) is factored M_x = L_x Q_x by Householder LQ and only the
// triangular L_x is kept, since the cuts need the right part only through
// L_{x+1} (its Gram matrix L L^T is never formed). Then, left to right, the
// centre C_x = G_x B_x (G_x: the truncated left part carried in) is multiplied
// by L_{x+1}; C_x L_{x+1} has the same left singular vectors as the centre in
// right-canonical gauge, and those are found by an LQ of C_x L_{x+1} followed
// by one-sided Jacobi on its triangular factor. The chi largest singular
// directions become the new site tensor and G_{x+1} = U^T C_x. No step squares
// a singular value, so FP32 resolves the kept directions to FP32 rounding.
//
// A second route (opt-in, TNMC_ROUTE_DM) reaches the same cut from the
// eigenvectors of the reduced density matrix rho_x = C_x N_{x+1} C_x^T, with
// N_{x+1} the right Gram matrix. It squares singular values, so in FP32 it
// resolves a kept direction only down to sqrt(eps) of the largest.
//
// Row MPO channels. The row factor prod_x psih(s_x, s_x+1) is carried on the
// bond as a channel k: site 0 has none; site 1 carries t = s_0; sites x >= 2
// carry (c, t) = (s_0, s_{x-1}) on periodic rows (ring) and t = s_{x-1} on open
// rows. The spin v at site x maps channel k to kn(x, k, v) with factor
// hf(x, k, v) = psih_{x-1}(t, v); the last site closes the ring with
// psih_{L-1}(v, s_0).
#pragma once

#include "common.cuh"
#include "fields.cuh"
#include "linalg.cuh"
#include <type_traits>

#include "tc_gemm.cuh"
#include "umma.cuh"
#include "arnet.cuh"


namespace tnmc {

// Sizes of the per-CTA workspace (all in elements of R unless noted).
struct WsLayout {
  int Mmax, Lmax, dmax, chimax, Dkmax, nmax;
  size_t off_phi, off_psih, off_psiv, off_E, off_N, off_G, off_G2, off_Gp, off_Y, off_C, off_Q, off_T1, off_M,
      off_rho, off_V, off_Rv, off_tmp, off_Mw, off_pan, off_Wb, total_R;
  size_t off_sold, off_snew, off_dims, total_bytes;  // bytes after the R region
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename R>
inline WsLayout make_layout(int Mmax, int Lmax, int dmax, int chimax) {
  WsLayout w;
  w.Mmax = Mmax; w.Lmax = Lmax; w.dmax = dmax; w.chimax = chimax;
  w.Dkmax = dmax * dmax;
  w.nmax = w.Dkmax * chimax;
  const size_t chi2 = (size_t)chimax * chimax;
  const size_t nm2 = (size_t)w.nmax * w.nmax;
  size_t o = 0;
  auto take = [&](size_t n) { size_t r = o; o = align_up(o + n, 32); return r; };
  w.off_phi = take((size_t)Mmax * Lmax * dmax);
  w.off_psih = take((size_t)Mmax * Lmax * dmax * dmax);
  w.off_psiv = take((size_t)Mmax * Lmax * dmax * dmax);
  w.off_E = take((size_t)Mmax * Lmax * dmax * chi2);
  w.off_N = take((size_t)(Lmax + 1) * nm2);
  w.off_G = take((size_t)chimax * w.nmax);
  w.off_G2 = take((size_t)chimax * w.nmax);
  w.off_Gp = take((size_t)w.Dkmax * chi2);
  w.off_Y = take((size_t)w.Dkmax * chi2);
  w.off_C = take((size_t)dmax * chimax * w.nmax);
  w.off_Q = take((size_t)dmax * chimax * w.nmax);
  w.off_T1 = take(nm2);
  w.off_M = take(nm2);
  w.off_rho = take((size_t)dmax * chimax * dmax * chimax);
  w.off_V = take((size_t)dmax * chimax * (dmax * chimax + 4));
  w.off_Rv = take((size_t)(Lmax + 1) * w.nmax);
  w.off_tmp = take((size_t)4 * w.nmax + 64);
  w.off_Mw = take((size_t)w.nmax * dmax * w.nmax);          // LQ input of the right sweep
  w.off_pan = take((size_t)32 * dmax * w.nmax);             // LQ panel when it is not in shared memory
  w.off_Wb = take((size_t)2 * w.nmax * 32 + 32 * 32);       // LQ trailing-update buffers
  w.total_R = o;
  size_t b = align_up(o * sizeof(R), 256);
  w.off_sold = b; b = align_up(b + (size_t)Mmax * Lmax, 256);
  w.off_snew = b; b = align_up(b + (size_t)Mmax * Lmax, 256);
  w.off_dims = b; b = align_up(b + sizeof(int) * (size_t)(Mmax + 1) * (Lmax + 1), 256);
  w.total_bytes = b;
  return w;
}

struct PhaseParams {
  const Group* groups;
  int n_groups;
  // explicit work list (n_items >= 0) or implicit colour class of a sweep (n_items < 0)
  const int* item_group;
  const int* item_chain;
  const int* item_slice;
  int n_items;
  int colour;
  const unsigned long long* sweep_ctr;   // implicit mode: axis = t % 3, step = 4 t + colour
  int axis;
  uint32_t step;
  uint64_t seed;
  double env_beta_factor;
  int write_back;
  int8_t* out_spins;  // [item][Lmax * Lmax]
  double* out_lq_new;
  double* out_lq_old;
  uint8_t* out_acc;
  int64_t* out_dE;
  unsigned int* acc_counter;          // [global chains]
  unsigned long long* event_counter;  // floor fallbacks (non-finite or empty conditionals)
  unsigned int* status;               // latched StatusBits (ST_NONFINITE), read by the next synchronising call
  double* out_logz;                   // logz mode: [item]
  int logz_only;
  int route;                          // ROUTE_LQ (LQ + one-sided Jacobi SVD) or ROUTE_DM (density matrix)
  size_t dyn_bytes;                   // dynamic shared memory of the launch
  int eig_smem;                       // 1: the (d chi)^2 eigenproblem lives in dynamic shared memory
  int jac_floor;                      // absolute convergence floor of the eigensolver (0 none, 1 eps^2 n, 2 eps)
  int gemm_mode;                      // FP32 path contractions: a GemmMode
  int umma_stage;                     // 1: dynamic shared memory holds the tcgen05 GEMM staging
  int proposal;                       // 0 tensor network, 1 learned network
  int n_prop;                         // tensor-network proposals per environment build (>= 1)
  const unsigned long long* proposal_ctr;  // implicit mode: proposal = net_every && t % net_every == net_every-1
  int net_every;
  NetLayout net;
  const float* net_W;
  float* net_ws;                      // per-CTA: cond, z, x buffers and compact spins
  size_t net_ws_stride;               // floats
  int net_Pmax;
  int record;                         // store accepted tensor-network slices for training
  float* rb_cond;                     // [slots][Cc][Pmax]
  int8_t* rb_spins;                   // [slots][Pmax]
  int* rb_meta;                       // [slots][2] = (m, Lc)
  unsigned long long* rb_counter;      // recording positions offered before this launch
  int rb_slots;
  // cache of environment stacks built for earlier held fields (one slot per chain, axis and slice):
  // CACHE_BUILD contracts every item's environments into its slot and records its fixed lines (no
  // sampling); CACHE_USE proposes every item from its slot; CACHE_SWEEP does so except on sweeps t with
  // cache_every > 0 and t mod cache_every = cache_every - 1, which contract afresh
  int gemm_tile;                      // CUDA-core GEMM tile of the float kernel: 0 64x64, 1 32x32, 2 128x64
  int cache_mode;
  int cache_every;
  char* cache;                        // [global chains][3][cache_lmax] slots of cache_stride bytes
  size_t cache_stride;
  int cache_lmax;
  size_t cache_dims_off;              // byte offsets inside a slot: environments at 0, then bond dims,
  size_t cache_meta_off;              // then (y0, x0, built)
  char* ws;
  size_t ws_stride;
  WsLayout lay;
};

enum Route : int { ROUTE_LQ = 0, ROUTE_DM = 1 };
enum CacheMode : int { CACHE_OFF = 0, CACHE_BUILD = 1, CACHE_USE = 2, CACHE_SWEEP = 3 };

template <typename R>
struct Ws {
  R *phi, *psih, *psiv, *E, *N, *G, *G2, *Gp, *Y, *C, *Q, *T1, *M, *rho, *V, *Rv, *tmp, *Mw, *pan, *Wb;
  int8_t *sold, *snew;
  int* dims;
  R* dyn;  // dynamic shared memory for the eigenproblem (nullptr: use global workspace)
  unsigned char* stage;  // tcgen05 GEMM staging in dynamic shared memory (nullptr: none)
};

template <typename R>
__device__ inline Ws<R> bind_ws(const PhaseParams& P) {
  char* base = P.ws + (size_t)blockIdx.x * P.ws_stride;
  R* r = reinterpret_cast<R*>(base);
  const WsLayout& L = P.lay;
  Ws<R> w;
  w.phi = r + L.off_phi; w.psih = r + L.off_psih; w.psiv = r + L.off_psiv; w.E = r + L.off_E;
  w.N = r + L.off_N; w.G = r + L.off_G; w.G2 = r + L.off_G2; w.Gp = r + L.off_Gp; w.Y = r + L.off_Y;
  w.C = r + L.off_C; w.Q = r + L.off_Q; w.T1 = r + L.off_T1; w.M = r + L.off_M; w.rho = r + L.off_rho;
  w.V = r + L.off_V; w.Rv = r + L.off_Rv; w.tmp = r + L.off_tmp;
  w.Mw = r + L.off_Mw; w.pan = r + L.off_pan; w.Wb = r + L.off_Wb;
  w.sold = reinterpret_cast<int8_t*>(base + L.off_sold);
  w.snew = reinterpret_cast<int8_t*>(base + L.off_snew);
  w.dims = reinterpret_cast<int*>(base + L.off_dims);
  w.dyn = nullptr;
  w.stage = nullptr;
  return w;
}

template <typename R>
struct SliceSmem {
  GemmSmem<R> g;
  TcGemmSmem tc;
  JacobiSmem<R> js;
  LqSmem<R> lq;
  int kr[132];   // columns k_x of the right factors L_x (LQ route)
  int tri[132];  // 1: L_x is lower triangular (it came from an LQ)
  int pn[16];    // nonzero columns of the product P_{k'} (LQ route)
  int jflag;     // rotation flag of the one-sided Jacobi
  UmmaCtl uctl;  // mbarrier and tensor-memory address of the tcgen05 GEMM
  R maxn2;       // largest squared row norm after the one-sided Jacobi
  double redd[32];
  long long redl[32];
  R redr[32];
  R W2[16];
  R hf[64];      // channel factor hf(x, k, v) of the current site, [k][v]
  int kn[64];    // next channel kn(x, k, v)
  double pt[8];
  double lscale;
  int choice;
};

__device__ inline int Dk_of(int x, int d, int ring) { return x == 0 ? 1 : (x == 1 ? d : (ring ? d * d : d)); }

// Non-last site x: factor of spin v given left channel k; *kn receives the right channel.
template <typename R>
__device__ inline R hfac(int x, int k, int v, int d, int ring, const R* psih_row, int* kn) {
  if (x == 0) { *kn = v; return R(1); }
  if (x == 1) { *kn = (ring ? k : 0) * d + v; return psih_row[((x - 1) * d + k) * d + v]; }
  const int c = k / d, t = k - c * d;
  *kn = c * d + v;
  return psih_row[((x - 1) * d + t) * d + v];
}
// Last site x = Lc - 1 >= 1: factor of spin v given left channel k.
template <typename R>
__device__ inline R hlast(int x, int k, int v, int d, int ring, const R* psih_row) {
  if (x == 1) {
    R f = psih_row[(0 * d + k) * d + v];
    if (ring) f *= psih_row[(1 * d + v) * d + k];
    return f;
  }
  const int c = k / d, t = k - c * d;
  R f = psih_row[((x - 1) * d + t) * d + v];
  if (ring) f *= psih_row[(x * d + v) * d + c];
  return f;
}

// ---------------------------------------------------------------- a1: weights
template <typename R>
__device__ void build_weights(const Group& g, const SliceGeom& s, const int8_t* spins, const int32_t* J, double beta,
                              const PhaseParams& P, Ws<R>& w, SliceSmem<R>& sm) {
  const int d = g.d, Lmax = P.lay.Lmax;
  const double b = beta * kJScale;
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  double lsc = 0.0;
  for (int e = threadIdx.x; e < s.m * s.Lc; e += kThreads) {
    const int r = e / s.Lc + 1, x = e % s.Lc;
    long long h[4];
    site_field(g, s, spins, J, r, x, h);
    long long hm = h[0];
    for (int v = 1; v < d; ++v) hm = h[v] > hm ? h[v] : hm;
    for (int v = 0; v < d; ++v) w.phi[((r - 1) * Lmax + x) * d + v] = (R)exp(b * (double)(h[v] - hm));
    lsc += b * (double)hm;
    const int idx = site_index(g, s, r, x);
    w.sold[(r - 1) * Lmax + x] = (int8_t)read_site(g, s, spins, r, x);
    // in-row bond (r, x) -> (r, x+1) (wrap on rings) and row bond (r, x) -> (r+1, x); the integer
    // energies are exact in double, so exp sees the same argument as for a scalar coupling
    for (int kind = 0; kind < 2; ++kind) {
      const bool present = kind == 0 ? ((x + 1 < s.Lc) || s.ring) : (r < s.m);
      R* out = (kind == 0 ? w.psih : w.psiv) + ((size_t)((r - 1) * Lmax + x) * d) * d;
      if (!present) {
        for (int t = 0; t < d * d; ++t) out[t] = R(1);
        continue;
      }
      const int ba = kind == 0 ? s.ca : s.ra;
      double mx = -1e300;
      for (int v = 0; v < d; ++v)
        for (int u = 0; u < d; ++u) {
          const double ex = (double)bond_energy(g, s, J, vol, idx, ba, v, u);
          mx = ex > mx ? ex : mx;
        }
      for (int v = 0; v < d; ++v)
        for (int u = 0; u < d; ++u) out[v * d + u] = (R)exp(b * ((double)bond_energy(g, s, J, vol, idx, ba, v, u) - mx));
      lsc += b * mx;
    }
  }
  lsc = block_sum(lsc, sm.redd);
  if (threadIdx.x == 0) sm.lscale = lsc;
  __syncthreads();
}

// Contractions of the environment pass: CUDA-core FMA, or tensor cores (3xTF32 / BF16) on the FP32 path:
// tcgen05.mma when the caller passes a free staging area in shared memory (the LQ route between its
// factorisations), else warp-level mma.sync with the same operand rounding. The factorisations (LQ,
// Jacobi) always run in the working precision on the CUDA cores.
// The tcgen05 engine is compiled only into its own kernel instance (TNMC_WITH_UMMA, slice_f32_umma.cu):
// a kernel that holds tensor-memory instructions is given one resident CTA per SM, so the default
// instances, which run two, carry none.
#ifndef TNMC_WITH_UMMA
#define TNMC_WITH_UMMA 0
#endif
template <typename R>
__device__ inline void gemm(const PhaseParams& P, SliceSmem<R>& sm, int M, int N, int K, R alpha, const R* A, int lda,
                            bool ta, const R* B, int ldb, bool tb, R beta, R* C, int ldc, bool b_lower = false,
                            unsigned char* stage = nullptr) {
  if constexpr (sizeof(R) == 4) {
    if (P.gemm_mode == GEMM_UMMA_TF32X3 || P.gemm_mode == GEMM_UMMA_BF16) {
#if TNMC_WITH_UMMA
      if (stage) {
        if (P.gemm_mode == GEMM_UMMA_BF16)
          cta_gemm_umma<UMMA_BF16>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, stage, sm.uctl, P.status);
        else
          cta_gemm_umma<UMMA_TF32X3>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, stage, sm.uctl, P.status);
        return;
      }
#endif
      cta_gemm_tc(P.gemm_mode == GEMM_UMMA_BF16 ? GEMM_BF16 : GEMM_TF32X3, M, N, K, alpha, A, lda, ta, B, ldb, tb,
                  beta, C, ldc, sm.tc);
      return;
    }
    if (P.gemm_mode != GEMM_FFMA) {
      cta_gemm_tc(P.gemm_mode, M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, sm.tc);
      return;
    }
  }
  cta_gemm<R>(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, sm.g, b_lower);
}

// ------------------------------------------------------------ a2: environments
// Row r (1-based) data pointers.
template <typename R>
struct RowView {
  const R* phi;   // [Lmax][d]
  const R* psih;  // [Lmax][d][d]
  const R* psiv;  // [Lmax][d][d] bond to the row below (r -> r+1); nullptr = none
};

template <typename R>
__device__ inline R* env_ptr(Ws<R>& w, const WsLayout& L, int r, int x, int v) {
  return w.E + (((size_t)(r - 1) * L.Lmax + x) * L.dmax + v) * (size_t)L.chimax * L.chimax;
}

// Density-matrix route (opt-in): build E_{r-1} from E_r using row r's factors and the row bond
// psiv_{r-1} (u = row r-1 spin). Returns the log of the norm divided out.
template <typename R>
__device__ double env_step_dm(const Group& g, const SliceGeom& s, int r, const PhaseParams& P, Ws<R>& w,
                           SliceSmem<R>& sm) {
  const WsLayout& L = P.lay;
  const int d = g.d, Lc = s.Lc, ring = s.ring, chi = g.chi, ldE = L.chimax;
  const R* phi = w.phi + (size_t)(r - 1) * L.Lmax * d;
  const R* psih = w.psih + (size_t)(r - 1) * L.Lmax * d * d;
  const R* psiv = w.psiv + (size_t)(r - 2) * L.Lmax * d * d;  // bond (r-1) -> r: [x][u][v]
  const int* dimr = w.dims + (size_t)(r - 1) * (L.Lmax + 1);
  int* dimn = w.dims + (size_t)(r - 2) * (L.Lmax + 1);
  const size_t nm2 = (size_t)L.nmax * L.nmax;
  auto wuv = [&](int x, int u, int v) -> R { return psiv[(x * d + u) * d + v] * phi[x * d + v]; };
  auto Nptr = [&](int x) { return w.N + (size_t)x * nm2; };

  // ---- right sweep: Gram matrices N_x of sites x..Lc-1 on the left bond of x
  TNMC_PROF_BEGIN(0);
  {
    const int x = Lc - 1;
    const int cx = dimr[x], Dk = Dk_of(x, d, ring), n = Dk * cx;
    R* f = w.tmp;  // [d][n]
    for (int e = threadIdx.x; e < d * n; e += kThreads) {
      const int u = e / n, ka = e % n, k = ka / cx, a = ka % cx;
      R acc = R(0);
      for (int v = 0; v < d; ++v) acc += wuv(x, u, v) * hlast(x, k, v, d, ring, psih) * env_ptr(w, L, r, x, v)[a * ldE];
      f[u * n + ka] = acc;
    }
    __syncthreads();
    R* N = Nptr(x);
    R loc = R(0);
    for (int e = threadIdx.x; e < n * n; e += kThreads) {
      const int i = e / n, j = e % n;
      R acc = R(0);
      for (int u = 0; u < d; ++u) acc += f[u * n + i] * f[u * n + j];
      N[e] = acc;
      if (i == j) loc = fmax(loc, acc);
    }
    const R mx = block_max(loc, sm.redr);
    const R inv = mx > R(0) ? R(1) / mx : R(1);
    for (int e = threadIdx.x; e < n * n; e += kThreads) N[e] *= inv;
    __syncthreads();
  }
  for (int x = Lc - 2; x >= 1; --x) {
    const int cx = dimr[x], cn = dimr[x + 1];
    const int Dk = Dk_of(x, d, ring), Dkn = Dk_of(x + 1, d, ring);
    const int n = Dk * cx, nn = Dkn * cn;
    const R* Nn = Nptr(x + 1);
    // M[k'][k2'] = A_{v(k')} Nn[k', k2'] A_{v(k2')}^T is symmetric in (k', k2') (Nn is), so only the
    // blocks k' <= k2' are formed: T1[k'][:, k2' >= k'] = A_{v(k')} Nn[k' rows, k2' >= k' columns]
    TNMC_PROF_BEGIN(8);
    for (int kp = 0; kp < Dkn; ++kp) {
      const int v = kp % d;
      gemm<R>(P, sm, cx, nn - kp * cn, cn, R(1), env_ptr(w, L, r, x, v), ldE, false,
                  Nn + (size_t)kp * cn * nn + (size_t)kp * cn, nn, false, R(0),
                  w.T1 + (size_t)kp * cx * nn + (size_t)kp * cn, nn);
    }
    // M[(k',a),(k2',a2)] = T1[k'][a, k2' block] A_{v(k2')}^T for k' <= k2'   ld = Dkn * cx
    const int ldm = Dkn * cx;
    for (int k2p = 0; k2p < Dkn; ++k2p) {
      const int v2 = k2p % d;
      gemm<R>(P, sm, (k2p + 1) * cx, cx, cn, R(1), w.T1 + (size_t)k2p * cn, nn, false, env_ptr(w, L, r, x, v2), ldE,
                  true, R(0), w.M + (size_t)k2p * cx, ldm);
    }
    TNMC_PROF_END(8);
    if (threadIdx.x < d * d) {
      const int v = threadIdx.x / d, v2 = threadIdx.x % d;
      R acc = R(0);
      for (int u = 0; u < d; ++u) acc += wuv(x, u, v) * wuv(x, u, v2);
      sm.W2[threadIdx.x] = acc;
    }
    // channel table of this site: factor and next channel of (k, v)
    if (threadIdx.x < Dk * d) {
      const int k = threadIdx.x / d, v = threadIdx.x % d;
      int kn;
      sm.hf[threadIdx.x] = hfac(x, k, v, d, ring, psih, &kn);
      sm.kn[threadIdx.x] = kn;
    }
    __syncthreads();
    TNMC_PROF_BEGIN(4);
    R* N = Nptr(x);
    // N_x[(k,a),(k2,a2)] = sum_{v,v2} W2(v,v2) hf(k,v) hf(k2,v2) M[(kn(k,v),a),(kn(k2,v2),a2)], with M
    // stored for block rows kn <= kn2 only (read transposed otherwise). Term t = v d + v2 of block
    // (k, k2) reads M at base + a * sa + a2 * sb.
    auto term = [&](int k, int k2, int t, R& coef, int& base, int& sa, int& sb) {
      const int v = t / d, v2 = t - v * d;
      const int kn = sm.kn[k * d + v], kn2 = sm.kn[k2 * d + v2];
      coef = sm.W2[t] * sm.hf[k * d + v] * sm.hf[k2 * d + v2];
      if (kn <= kn2) { base = kn * cx * ldm + kn2 * cx; sa = ldm; sb = 1; }
      else { base = kn2 * cx * ldm + kn * cx; sa = 1; sb = ldm; }
    };
    const int dd = d * d;
    // the diagonal first: its largest entry normalises N_x as it is written
    R loc = R(0);
    for (int i = threadIdx.x; i < n; i += kThreads) {
      const int k = i / cx, a = i - k * cx;
      R acc = R(0);
      for (int t = 0; t < dd; ++t) {
        R coef; int base, sa, sb;
        term(k, k, t, coef, base, sa, sb);
        acc += coef * w.M[(size_t)base + (size_t)a * (sa + sb)];
      }
      loc = fmax(loc, acc);
    }
    const R mx = block_max(loc, sm.redr);
    const R inv = mx > R(0) ? R(1) / mx : R(1);
    // N_x is symmetric: blocks k <= k2 are computed and mirrored. For d = 2 a thread takes four
    // entries at a time and issues all their loads before any store (M and N share the workspace,
    // so the compiler would otherwise wait for each entry's loads in turn).
    auto combine4 = [&]() {
      constexpr int T = 4, U = 4;
      for (int k = 0; k < Dk; ++k)
        for (int k2 = k; k2 < Dk; ++k2) {
          R coef[T];
          int base[T], sa[T], sb[T];
#pragma unroll
          for (int t = 0; t < T; ++t) term(k, k2, t, coef[t], base[t], sa[t], sb[t]);
          for (int e0 = threadIdx.x; e0 < cx * cx; e0 += U * kThreads) {
            R mv[U][T];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int e = e0 + u * kThreads, a = e / cx, a2 = e - a * cx;
              if (e < cx * cx && (k < k2 || a2 >= a)) {
#pragma unroll
                for (int t = 0; t < T; ++t) mv[u][t] = w.M[(size_t)base[t] + (size_t)a * sa[t] + (size_t)a2 * sb[t]];
              }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int e = e0 + u * kThreads, a = e / cx, a2 = e - a * cx;
              if (e < cx * cx && (k < k2 || a2 >= a)) {
                R acc = R(0);
#pragma unroll
                for (int t = 0; t < T; ++t) acc += coef[t] * mv[u][t];
                acc *= inv;
                const int i = k * cx + a, j = k2 * cx + a2;
                N[(size_t)i * n + j] = acc;
                N[(size_t)j * n + i] = acc;
              }
            }
          }
        }
    };
    if (d == 2) {
      combine4();
    } else {
      for (int k = 0; k < Dk; ++k)
        for (int k2 = k; k2 < Dk; ++k2)
          for (int e = threadIdx.x; e < cx * cx; e += kThreads) {
            const int a = e / cx, a2 = e - a * cx;
            if (k == k2 && a2 < a) continue;
            R acc = R(0);
            for (int t = 0; t < dd; ++t) {
              R coef; int base, sa, sb;
              term(k, k2, t, coef, base, sa, sb);
              acc += coef * w.M[(size_t)base + (size_t)a * sa + (size_t)a2 * sb];
            }
            acc *= inv;
            const int i = k * cx + a, j = k2 * cx + a2;
            N[(size_t)i * n + j] = acc;
            N[(size_t)j * n + i] = acc;
          }
    }
    __syncthreads();
    TNMC_PROF_END(4);
  }

  TNMC_PROF_END(0);
  // ---- left sweep with truncation
  TNMC_PROF_BEGIN(1);
  double lognorm = 0.0;
  R* G = w.G;
  R* G2 = w.G2;
  if (threadIdx.x == 0) { G[0] = R(1); dimn[0] = 1; }
  __syncthreads();
  int cp = 1;  // rows of G (new left bond)
  for (int x = 0; x < Lc - 1; ++x) {
    const int cx = dimr[x], cn = dimr[x + 1];
    const int Dk = Dk_of(x, d, ring), Dkn = Dk_of(x + 1, d, ring);
    const int n = Dk * cx, nn = Dkn * cn;
    TNMC_PROF_BEGIN(9);
    // G'[k'][i][a] = sum_{k : kn(k, v(k')) = k'} hf(k, v(k')) G[i][k*cx + a]
    for (int e = threadIdx.x; e < Dkn * cp * cx; e += kThreads) {
      const int kp = e / (cp * cx), ia = e % (cp * cx), i = ia / cx, a = ia % cx;
      const int v = kp % d;
      R acc = R(0);
      for (int k = 0; k < Dk; ++k) {
        int kn;
        const R f = hfac(x, k, v, d, ring, psih, &kn);
        if (kn == kp) acc += f * G[(size_t)i * n + k * cx + a];
      }
      w.Gp[(size_t)kp * cp * cx + ia] = acc;
    }
    __syncthreads();
    // Y[k'] = G'[k'] A_{v(k')}   (cp x cn). The centre is C_u[i][(k', b)] = w(u, v(k')) Y[k'][i][b].
    for (int kp = 0; kp < Dkn; ++kp)
      gemm<R>(P, sm, cp, cn, cx, R(1), w.Gp + (size_t)kp * cp * cx, cx, false, env_ptr(w, L, r, x, kp % d), ldE, false,
                  R(0), w.Y + (size_t)kp * cp * cn, cn);
    TNMC_PROF_END(9);
    const int nd = d * cp;
    int keep = chi;
    if (keep > nd) keep = nd;
    if (keep > nn) keep = nn;
    R* E0 = env_ptr(w, L, r - 1, x, 0);
    const size_t vstride = (size_t)L.chimax * L.chimax;
    if (keep == nd) {
      // nothing to cut: identity gauge, E tensor = I, G_new = stacked C_u
      for (int e = threadIdx.x; e < nd * keep; e += kThreads) {
        const int row = e / keep, j = e % keep, u = row / cp, i = row % cp;
        E0[u * vstride + (size_t)i * ldE + j] = (row == j) ? R(1) : R(0);
      }
      for (int e = threadIdx.x; e < nd * nn; e += kThreads) {
        const int row = e / nn, col = e % nn, u = row / cp, i = row % cp;
        const int kp = col / cn, bb = col % cn;
        G2[e] = wuv(x, u, kp % d) * w.Y[((size_t)kp * cp + i) * cn + bb];
      }
    } else {
      // rho[(u,i),(u2,i2)] = sum_{v,v2} w(u,v) w(u2,v2) Zt[v][v2][i][i2],
      // Zt[v][v2] = sum over channels k' of spin v and k2' of spin v2 of Y[k'] N[k', k2'] Y[k2']^T
      const R* Nn = Nptr(x + 1);
      R* Pv = w.Q;   // [d][cp][nn]
      R* Zt = w.C;   // [d][d][cp][cp]
      TNMC_PROF_BEGIN(10);
      for (int v = 0; v < d; ++v) {
        bool first = true;
        for (int kp = v; kp < Dkn; kp += d) {
          gemm<R>(P, sm, cp, nn, cn, R(1), w.Y + (size_t)kp * cp * cn, cn, false, Nn + (size_t)kp * cn * nn, nn, false,
                      first ? R(0) : R(1), Pv + (size_t)v * cp * nn, nn);
          first = false;
        }
      }
      for (int v = 0; v < d; ++v)
        for (int v2 = v; v2 < d; ++v2) {
          bool first = true;
          for (int k2p = v2; k2p < Dkn; k2p += d) {
            gemm<R>(P, sm, cp, cp, cn, R(1), Pv + (size_t)v * cp * nn + (size_t)k2p * cn, nn, false,
                        w.Y + (size_t)k2p * cp * cn, cn, true, first ? R(0) : R(1),
                        Zt + (size_t)(v * d + v2) * cp * cp, cp);
            first = false;
          }
        }
      // rho is symmetric: blocks (u, u2 >= u) are computed and mirrored, so it is exactly symmetric
      TNMC_PROF_END(10);
      TNMC_PROF_BEGIN(7);
      if (threadIdx.x < d * d) sm.W2[threadIdx.x] = wuv(x, threadIdx.x / d, threadIdx.x % d);   // w(u, v)
      __syncthreads();
      for (int u = 0; u < d; ++u)
        for (int u2 = u; u2 < d; ++u2)
          for (int e = threadIdx.x; e < cp * cp; e += kThreads) {
            const int i = e / cp, i2 = e - i * cp;
            if (u == u2 && i2 < i) continue;
            R acc = R(0);
            for (int v = 0; v < d; ++v)
              for (int v2 = 0; v2 < d; ++v2) {
                const R z = v <= v2 ? Zt[((size_t)(v * d + v2) * cp + i) * cp + i2]
                                    : Zt[((size_t)(v2 * d + v) * cp + i2) * cp + i];
                acc += sm.W2[u * d + v] * sm.W2[u2 * d + v2] * z;
              }
            const int row = u * cp + i, col = u2 * cp + i2;
            w.rho[(size_t)row * nd + col] = acc;
            w.rho[(size_t)col * nd + row] = acc;
          }
      __syncthreads();
      TNMC_PROF_END(7);
      // the matrix in shared memory when it fits (padded by one column); eigenvectors in the workspace
      const int lda = w.dyn ? nd + 1 : nd;
      R* JA = w.dyn ? w.dyn : w.rho;
      R* JV = w.V;
      if (w.dyn) {
        for (int e = threadIdx.x; e < nd * nd; e += kThreads) JA[(e / nd) * lda + e % nd] = w.rho[e];
        __syncthreads();
      }
      TNMC_PROF_BEGIN(2);
      const int ldv = (nd + 3) & ~3;
      const int nsw = cta_jacobi_eig_fused<R>(nd, JA, lda, JV, ldv, sizeof(R) == 8 ? 30 : 20, sm.js, sm.redr,
                                              P.jac_floor);
      TNMC_PROF_END(2);
#ifdef TNMC_PROFILE
      if (threadIdx.x == 0) { atomicAdd(&tnmc_prof[5], (unsigned long long)nsw); atomicAdd(&tnmc_prof[6], 1ull); }
#else
      (void)nsw;
#endif
      TNMC_PROF_BEGIN(11);
      int* rank = reinterpret_cast<int*>(w.tmp);
      cta_rank_desc<R>(nd, JA, lda, rank);
      // U[(u,i), j] = eigenvector with rank j (rows of JV are eigenvectors)
      for (int e = threadIdx.x; e < nd * nd; e += kThreads) {
        const int k = e / nd, row = e % nd;
        const int j = rank[k];
        if (j < keep) {
          const int u = row / cp, i = row % cp;
          E0[u * vstride + (size_t)i * ldE + j] = JV[(size_t)k * ldv + row];
        }
      }
      __syncthreads();
      // G_new[j][(k', b)] = sum_i Ut_{v(k')}[i][j] Y[k'][i][b],  Ut_v[i][j] = sum_u w(u, v) U[(u,i), j]
      R* Ut = w.Gp;  // [d][cp][keep]
      for (int e = threadIdx.x; e < d * cp * keep; e += kThreads) {
        const int v = e / (cp * keep), rem = e % (cp * keep), i = rem / keep, j = rem % keep;
        R acc = R(0);
        for (int u = 0; u < d; ++u) acc += wuv(x, u, v) * E0[u * vstride + (size_t)i * ldE + j];
        Ut[e] = acc;
      }
      __syncthreads();
      for (int kp = 0; kp < Dkn; ++kp)
        gemm<R>(P, sm, keep, cn, cp, R(1), Ut + (size_t)(kp % d) * cp * keep, keep, true, w.Y + (size_t)kp * cp * cn,
                    cn, false, R(0), G2 + (size_t)kp * cn, nn);
      TNMC_PROF_END(11);
    }
    __syncthreads();
    // normalise the carried centre
    R loc = R(0);
    for (int e = threadIdx.x; e < keep * nn; e += kThreads) loc += G2[e] * G2[e];
    const R ss = block_sum(loc, sm.redr);
    const R nrm = sqrt(ss);
    const R inv = nrm > R(0) ? R(1) / nrm : R(1);
    for (int e = threadIdx.x; e < keep * nn; e += kThreads) G2[e] *= inv;
    if (threadIdx.x == 0) dimn[x + 1] = keep;
    if (threadIdx.x == 0) lognorm += nrm > R(0) ? log((double)nrm) : 0.0;
    R* t = G; G = G2; G2 = t;
    cp = keep;
    __syncthreads();
  }
  {
    const int x = Lc - 1;
    const int cx = dimr[x], Dk = Dk_of(x, d, ring), n = Dk * cx;
    // a[(k,a)][u] = sum_v A_v[a][0] w(u, v) hl(k, v);  C[i][u] = G[i] . a[:, u]
    R* av = w.tmp;
    for (int e = threadIdx.x; e < n * d; e += kThreads) {
      const int ka = e / d, u = e % d, k = ka / cx, a = ka % cx;
      R acc = R(0);
      for (int v = 0; v < d; ++v) acc += env_ptr(w, L, r, x, v)[a * ldE] * wuv(x, u, v) * hlast(x, k, v, d, ring, psih);
      av[e] = acc;
    }
    __syncthreads();
    R* E0 = env_ptr(w, L, r - 1, x, 0);
    const size_t vstride = (size_t)L.chimax * L.chimax;
    R loc = R(0);
    R* Cl = w.Q;
    for (int e = threadIdx.x; e < cp * d; e += kThreads) {
      const int i = e / d, u = e % d;
      R acc = R(0);
      for (int ka = 0; ka < n; ++ka) acc += G[(size_t)i * n + ka] * av[ka * d + u];
      Cl[e] = acc;
      loc += acc * acc;
    }
    const R ss = block_sum(loc, sm.redr);
    const R nrm = sqrt(ss);
    const R inv = nrm > R(0) ? R(1) / nrm : R(1);
    for (int e = threadIdx.x; e < cp * d; e += kThreads) {
      const int i = e / d, u = e % d;
      E0[u * vstride + (size_t)i * ldE + 0] = Cl[e] * inv;
    }
    if (threadIdx.x == 0) dimn[Lc] = 1;
    if (threadIdx.x == 0) lognorm += nrm > R(0) ? log((double)nrm) : 0.0;
    __syncthreads();
  }
  TNMC_PROF_END(1);
  return lognorm;
}

// Rotation floor of the one-sided Jacobi relative to the largest row norm: rows below it are zero at
// the working precision (far below its rounding level) and are dropped from U.
template <typename R> struct kJacobiFloor { static constexpr R v = R(1e-10); };
template <> struct kJacobiFloor<double> { static constexpr double v = 1e-26; };

// Normalise the n x k block X (leading dimension ld) by its largest magnitude (the scale of a
// right factor is irrelevant to the cuts, which depend only on singular directions).
template <typename R>
__device__ inline void normalise_block(R* X, int n, int k, int ld, SliceSmem<R>& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R loc = R(0);
  for (int i = warp; i < n; i += kWarps)
    for (int j = lane; j < k; j += 32) loc = fmax(loc, fabs(X[(size_t)i * ld + j]));
  const R mx = block_max(loc, sm.redr);
  const R inv = mx > R(0) ? R(1) / mx : R(1);
  for (int i = warp; i < n; i += kWarps)
    for (int j = lane; j < k; j += 32) X[(size_t)i * ld + j] *= inv;
  __syncthreads();
}

// LQ route: build E_{r-1} from E_r (row r's factors and the row bond psiv_{r-1}, u = row r-1 spin)
// with the canonical SVD cut. Returns the log of the norm divided out.
template <typename R>
__device__ double env_step_lq(const Group& g, const SliceGeom& s, int r, const PhaseParams& P, Ws<R>& w,
                              SliceSmem<R>& sm) {
  const WsLayout& L = P.lay;
  const int d = g.d, Lc = s.Lc, ring = s.ring, chi = g.chi, ldE = L.chimax;
  const R* phi = w.phi + (size_t)(r - 1) * L.Lmax * d;
  const R* psih = w.psih + (size_t)(r - 1) * L.Lmax * d * d;
  const R* psiv = w.psiv + (size_t)(r - 2) * L.Lmax * d * d;  // bond (r-1) -> r: [x][u][v]
  const int* dimr = w.dims + (size_t)(r - 1) * (L.Lmax + 1);
  int* dimn = w.dims + (size_t)(r - 2) * (L.Lmax + 1);
  const int ldL = L.nmax;
  auto wuv = [&](int x, int u, int v) -> R { return psiv[(x * d + u) * d + v] * phi[x * d + v]; };
  auto Lp = [&](int x) { return w.N + (size_t)x * L.nmax * L.nmax; };
  // staging buffers of the factorisations: dynamic shared memory when they fit, else the workspace
  const size_t dyn_elems = w.dyn ? P.dyn_bytes / sizeof(R) : 0;
  R* Wb = w.Wb;
  R* Wb2 = w.Wb + (size_t)L.nmax * 32;
  R* Sb = w.Wb + (size_t)2 * L.nmax * 32;
  auto lq = [&](int n, int m, R* A, int lda) {
    R* pan = ((size_t)kLqPanel * m <= dyn_elems) ? w.dyn : w.pan;
    cta_lq<R>(n, m, A, lda, pan, Wb, Wb2, Sb, sm.lq, sm.g);
  };

  // ---- right sweep: L_x with L_x L_x^T = M_x M_x^T, M_x = B_x L_{x+1}
  TNMC_PROF_BEGIN(0);
  {
    const int x = Lc - 1;
    const int cx = dimr[x], Dk = Dk_of(x, d, ring), n = Dk * cx;
    R* Mw = w.Mw;  // [n][d]
    for (int e = threadIdx.x; e < n * d; e += kThreads) {
      const int ka = e / d, u = e % d, k = ka / cx, a = ka % cx;
      R acc = R(0);
      for (int v = 0; v < d; ++v) acc += wuv(x, u, v) * hlast(x, k, v, d, ring, psih) * env_ptr(w, L, r, x, v)[a * ldE];
      Mw[e] = acc;
    }
    __syncthreads();
    int kx = d;
    if (d > n) { lq(n, d, Mw, d); kx = n; }
    R* Lx = Lp(x);
    for (int e = threadIdx.x; e < n * kx; e += kThreads) Lx[(size_t)(e / kx) * ldL + e % kx] = Mw[(size_t)(e / kx) * d + e % kx];
    if (threadIdx.x == 0) { sm.kr[x] = kx; sm.tri[x] = d > n ? 1 : 0; }
    __syncthreads();
    normalise_block(Lx, n, kx, ldL, sm);
  }
  for (int x = Lc - 2; x >= 1; --x) {
    const int cx = dimr[x], cn = dimr[x + 1];
    const int Dk = Dk_of(x, d, ring), Dkn = Dk_of(x + 1, d, ring);
    const int n = Dk * cx;
    const int kk = sm.kr[x + 1];
    const R* Ln = Lp(x + 1);
    // P_{k'} = A_{v(k')} L_{x+1}[rows of channel k'] (cx x kk). A lower-triangular L_{x+1} makes
    // the rows of channel k' zero beyond column (k' + 1) cn, and P_{k'} with them.
    const int tri = sm.tri[x + 1];
    TNMC_PROF_BEGIN(8);
    R* Pb = w.T1;
    for (int kp = 0; kp < Dkn; ++kp) {
      int np = kk;
      if (tri && (kp + 1) * cn < np) np = (kp + 1) * cn;
      gemm<R>(P, sm, cx, np, cn, R(1), env_ptr(w, L, r, x, kp % d), ldE, false, Ln + (size_t)kp * cn * ldL, ldL, false,
              R(0), Pb + (size_t)kp * cx * kk, kk, false, w.stage);
      if (threadIdx.x == 0) sm.pn[kp] = np;
    }
    TNMC_PROF_END(8);
    if (threadIdx.x < Dk * d) {
      const int k = threadIdx.x / d, v = threadIdx.x % d;
      int kn;
      sm.hf[threadIdx.x] = hfac(x, k, v, d, ring, psih, &kn);
      sm.kn[threadIdx.x] = kn;
    }
    if (threadIdx.x < d * d) sm.W2[threadIdx.x] = wuv(x, threadIdx.x / d, threadIdx.x % d);
    __syncthreads();
    // M_x[(k, a)][(u, j)] = sum_v w(u, v) hf(k, v) P_{kn(k, v)}[a][j]. On ring rows with a triangular
    // L_{x+1} the channel k = (c, t) maps to kn = (c, v), so the rows of block c are zero beyond
    // column j = (c + 1) d cn: with the columns ordered by blocks of B = d cn values of j (all u of a
    // block together), the rows form a staircase that the LQ exploits. The column order does not
    // change L_x L_x^T = M_x M_x^T.
    const int mcols = d * kk;
    const bool stair = ring && tri;
    const int B = d * cn;
    R* Mw = w.Mw;
    // column -> (u, j) of M_x, once per site (staircase order on ring rows with a triangular L_{x+1})
    int* colj = reinterpret_cast<int*>(w.Wb);
    int* colu = colj + mcols;
    for (int col = threadIdx.x; col < mcols; col += kThreads) {
      int u, j;
      if (stair) {
        const int jb = col / (d * B), rem = col - jb * d * B;
        const int wb = (kk - jb * B) < B ? (kk - jb * B) : B;
        u = rem / wb;
        j = jb * B + (rem - u * wb);
      } else {
        u = col / kk;
        j = col - u * kk;
      }
      colj[col] = j;
      colu[col] = u;
    }
    __syncthreads();
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int row = warp; row < n; row += kWarps) {
        const int k = row / cx, a = row - k * cx;
        int knv[4];
        R hv[4];
        int lim[4];
        for (int v = 0; v < d; ++v) {
          knv[v] = sm.kn[k * d + v];
          hv[v] = sm.hf[k * d + v];
          lim[v] = sm.pn[knv[v]];
        }
        R* out = Mw + (size_t)row * mcols;
        for (int col = lane; col < mcols; col += 32) {
          const int j = colj[col], u = colu[col];
          R acc = R(0);
          for (int v = 0; v < d; ++v)
            if (j < lim[v]) acc += sm.W2[u * d + v] * hv[v] * Pb[((size_t)knv[v] * cx + a) * kk + j];
          out[col] = acc;
        }
      }
    }
    __syncthreads();
    TNMC_PROF_BEGIN(4);
    int kx = mcols;
    if (mcols > n) {
      R* pan = ((size_t)kLqPanel * mcols <= dyn_elems) ? w.dyn : w.pan;
      if (stair) cta_lq<R>(n, mcols, Mw, mcols, pan, Wb, Wb2, Sb, sm.lq, sm.g, (Dk / d) * cx, d * B);
      else cta_lq<R>(n, mcols, Mw, mcols, pan, Wb, Wb2, Sb, sm.lq, sm.g);
      kx = n;
    }
    TNMC_PROF_END(4);
    R* Lx = Lp(x);
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int i = warp; i < n; i += kWarps)
        for (int j = lane; j < kx; j += 32) Lx[(size_t)i * ldL + j] = Mw[(size_t)i * mcols + j];
    }
    if (threadIdx.x == 0) sm.tri[x] = mcols > n ? 1 : 0;
    if (threadIdx.x == 0) sm.kr[x] = kx;
    __syncthreads();
    normalise_block(Lx, n, kx, ldL, sm);
  }
  TNMC_PROF_END(0);

  // ---- left sweep with truncation
  TNMC_PROF_BEGIN(1);
  double lognorm = 0.0;
  R* G = w.G;
  R* G2 = w.G2;
  if (threadIdx.x == 0) { G[0] = R(1); dimn[0] = 1; }
  __syncthreads();
  int cp = 1;  // rows of G (new left bond)
  for (int x = 0; x < Lc - 1; ++x) {
    const int cx = dimr[x], cn = dimr[x + 1];
    const int Dk = Dk_of(x, d, ring), Dkn = Dk_of(x + 1, d, ring);
    const int n = Dk * cx, nn = Dkn * cn;
    const int kk = sm.kr[x + 1];
    TNMC_PROF_BEGIN(9);
    // G'[k'][i][a] = sum_{k : kn(k, v(k')) = k'} hf(k, v(k')) G[i][k*cx + a]
    if (threadIdx.x < Dk * d) {
      const int k = threadIdx.x / d, v = threadIdx.x % d;
      int kn;
      sm.hf[threadIdx.x] = hfac(x, k, v, d, ring, psih, &kn);
      sm.kn[threadIdx.x] = kn;
    }
    if (threadIdx.x < d * d) sm.W2[threadIdx.x] = wuv(x, threadIdx.x / d, threadIdx.x % d);
    __syncthreads();
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int rowp = warp; rowp < Dkn * cp; rowp += kWarps) {
        const int kp = rowp / cp, i = rowp - kp * cp, v = kp % d;
        R* out = w.Gp + (size_t)kp * cp * cx + (size_t)i * cx;
        for (int a = lane; a < cx; a += 32) {
          R acc = R(0);
          for (int k = 0; k < Dk; ++k)
            if (sm.kn[k * d + v] == kp) acc += sm.hf[k * d + v] * G[(size_t)i * n + k * cx + a];
          out[a] = acc;
        }
      }
    }
    __syncthreads();
    // Y[k'] = G'[k'] A_{v(k')}   (cp x cn)
    for (int kp = 0; kp < Dkn; ++kp)
      gemm<R>(P, sm, cp, cn, cx, R(1), w.Gp + (size_t)kp * cp * cx, cx, false, env_ptr(w, L, r, x, kp % d), ldE, false,
              R(0), w.Y + (size_t)kp * cp * cn, cn, false, w.stage);
    // centre C[(u, i)][(k', b)] = w(u, v(k')) Y[k'][i][b]   (nd x nn)
    const int nd = d * cp;
    R* C = w.C;
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int row = warp; row < nd; row += kWarps) {
        const int u = row / cp, i = row - u * cp;
        for (int kp = 0; kp < Dkn; ++kp) {
          const R wv = sm.W2[u * d + kp % d];
          const R* y = w.Y + ((size_t)kp * cp + i) * cn;
          R* out = C + (size_t)row * nn + (size_t)kp * cn;
          for (int bb = lane; bb < cn; bb += 32) out[bb] = wv * y[bb];
        }
      }
    }
    __syncthreads();
    TNMC_PROF_END(9);
    int keep = chi;
    if (keep > nd) keep = nd;
    if (keep > kk) keep = kk;
    R* E0 = env_ptr(w, L, r - 1, x, 0);
    const size_t vstride = (size_t)L.chimax * L.chimax;
    if (keep == nd) {
      // nothing to cut: identity gauge, E tensor = I, G_new = C
      for (int e = threadIdx.x; e < nd * keep; e += kThreads) {
        const int row = e / keep, j = e % keep, u = row / cp, i = row % cp;
        E0[u * vstride + (size_t)i * ldE + j] = (row == j) ? R(1) : R(0);
      }
      for (int e = threadIdx.x; e < nd * nn; e += kThreads) G2[e] = C[e];
    } else {
      // C' = C L_{x+1} (nd x kk): the centre in right-canonical gauge up to an orthogonal factor
      TNMC_PROF_BEGIN(10);
      R* Cp = w.Q;
      gemm<R>(P, sm, nd, kk, nn, R(1), C, nn, false, Lp(x + 1), ldL, false, R(0), Cp, kk, sm.tri[x + 1] != 0,
              w.stage);
      int kx = kk;
      if (kk > nd) { lq(nd, kk, Cp, kk); kx = nd; }
      TNMC_PROF_END(10);
      // Z = X^T (rows: the kx columns of X = C' or its L factor; length nd)
      TNMC_PROF_BEGIN(7);
      const int ldz = nd + 4;
      const size_t zbytes = (size_t)kx * ldz * sizeof(R);
      R* Z = (w.dyn && zbytes <= P.dyn_bytes) ? w.dyn : w.V;
      for (int e = threadIdx.x; e < kx * nd; e += kThreads) {
        const int j = e / nd, row = e - j * nd;
        Z[(size_t)j * ldz + row] = Cp[(size_t)row * kk + j];
      }
      __syncthreads();
      TNMC_PROF_END(7);
      TNMC_PROF_BEGIN(2);
      R* nrm2 = w.tmp;
      int* rank = reinterpret_cast<int*>(w.tmp + L.nmax + 32);
      const R tol = sqrt((R)nd) * Eps<R>::v;
      const int nsw = cta_onesided_jacobi<R>(kx, nd, Z, ldz, nrm2, &sm.maxn2, 40, tol, kJacobiFloor<R>::v, &sm.jflag,
                                             sm.redr);
      TNMC_PROF_END(2);
#ifdef TNMC_PROFILE
      if (threadIdx.x == 0) { atomicAdd(&tnmc_prof[5], (unsigned long long)nsw); atomicAdd(&tnmc_prof[6], 1ull); }
#else
      (void)nsw;
#endif
      TNMC_PROF_BEGIN(11);
      cta_rank_desc_vec<R>(kx, nrm2, rank);
      // U[(u, i)][rank j] = z_j / |z_j| for the keep largest. A row at or below the Jacobi's rotation
      // floor was not orthogonalised and gives a zero column (its singular value is zero at the
      // working precision). The floor sits far below the rounding level: dropping rows at the
      // rounding level itself (eps of the largest) measurably worsens log q at L = 32 in FP32.
      const R fl = kJacobiFloor<R>::v * kJacobiFloor<R>::v * sm.maxn2 * R(1.0001);
      R* U0 = w.Q;                          // [nd][keep] (C' is dead once Z holds it)
      R* U1 = w.Q + (size_t)nd * keep;      // [nd][keep]
      R* S = w.T1;                          // [keep][keep]
      for (int e = threadIdx.x; e < kx * nd; e += kThreads) {
        const int j = e / nd, row = e - j * nd;
        const int rj = rank[j];
        if (rj < keep) {
          const R nr = nrm2[j];
          const R inv = nr > fl ? R(1) / sqrt(nr) : R(0);
          U0[(size_t)row * keep + rj] = Z[(size_t)j * ldz + row] * inv;
        }
      }
      __syncthreads();
      // The Jacobi stops once every pair is orthogonal to within its tolerance, so U is orthonormal
      // only to that level, and U U^T would not be a projector. One Newton-Schulz step
      // U <- U (3 I - U^T U) / 2 keeps the span and squares the departure from orthonormality.
      cta_gemm<R>(keep, keep, nd, R(1), U0, keep, true, U0, keep, false, R(0), S, keep, sm.g);
      for (int e = threadIdx.x; e < keep * keep; e += kThreads)
        S[e] = (e / keep == e % keep ? R(1.5) : R(0)) - R(0.5) * S[e];
      __syncthreads();
      cta_gemm<R>(nd, keep, keep, R(1), U0, keep, false, S, keep, false, R(0), U1, keep, sm.g);
      for (int e = threadIdx.x; e < nd * keep; e += kThreads) {
        const int row = e / keep, j = e - row * keep, u = row / cp, i = row - u * cp;
        E0[u * vstride + (size_t)i * ldE + j] = U1[e];
      }
      // G_new = U^T C   (keep x nn)
      gemm<R>(P, sm, keep, nn, nd, R(1), U1, keep, true, C, nn, false, R(0), G2, nn, false, w.stage);
      TNMC_PROF_END(11);
    }
    __syncthreads();
    // normalise the carried centre
    R loc = R(0);
    for (int e = threadIdx.x; e < keep * nn; e += kThreads) loc += G2[e] * G2[e];
    const R ss = block_sum(loc, sm.redr);
    const R nrm = sqrt(ss);
    const R inv = nrm > R(0) ? R(1) / nrm : R(1);
    for (int e = threadIdx.x; e < keep * nn; e += kThreads) G2[e] *= inv;
    if (threadIdx.x == 0) dimn[x + 1] = keep;
    if (threadIdx.x == 0) lognorm += nrm > R(0) ? log((double)nrm) : 0.0;
    R* t = G; G = G2; G2 = t;
    cp = keep;
    __syncthreads();
  }
  {
    const int x = Lc - 1;
    const int cx = dimr[x], Dk = Dk_of(x, d, ring), n = Dk * cx;
    // a[(k,a)][u] = sum_v A_v[a][0] w(u, v) hl(k, v);  C[i][u] = G[i] . a[:, u]
    R* av = w.tmp;
    for (int e = threadIdx.x; e < n * d; e += kThreads) {
      const int ka = e / d, u = e % d, k = ka / cx, a = ka % cx;
      R acc = R(0);
      for (int v = 0; v < d; ++v) acc += env_ptr(w, L, r, x, v)[a * ldE] * wuv(x, u, v) * hlast(x, k, v, d, ring, psih);
      av[e] = acc;
    }
    __syncthreads();
    R* E0 = env_ptr(w, L, r - 1, x, 0);
    const size_t vstride = (size_t)L.chimax * L.chimax;
    R loc = R(0);
    R* Cl = w.Q;
    for (int e = threadIdx.x; e < cp * d; e += kThreads) {
      const int i = e / d, u = e % d;
      R acc = R(0);
      for (int ka = 0; ka < n; ++ka) acc += G[(size_t)i * n + ka] * av[ka * d + u];
      Cl[e] = acc;
      loc += acc * acc;
    }
    const R ss = block_sum(loc, sm.redr);
    const R nrm = sqrt(ss);
    const R inv = nrm > R(0) ? R(1) / nrm : R(1);
    for (int e = threadIdx.x; e < cp * d; e += kThreads) {
      const int i = e / d, u = e % d;
      E0[u * vstride + (size_t)i * ldE + 0] = Cl[e] * inv;
    }
    if (threadIdx.x == 0) dimn[Lc] = 1;
    if (threadIdx.x == 0) lognorm += nrm > R(0) ? log((double)nrm) : 0.0;
    __syncthreads();
  }
  TNMC_PROF_END(1);
  return lognorm;
}

// Closing contraction of row 1 with E_1 (physical index summed): log of the scalar.
template <typename R>
__device__ double close_row1(const Group& g, const SliceGeom& s, const PhaseParams& P, Ws<R>& w, SliceSmem<R>& sm) {
  const WsLayout& L = P.lay;
  const int d = g.d, Lc = s.Lc, ring = s.ring, ldE = L.chimax;
  const R* phi = w.phi;
  const R* psih = w.psih;
  const int* dim1 = w.dims;
  R* ell = w.Rv;
  R* nxt = w.Rv + L.nmax;
  if (threadIdx.x == 0) ell[0] = R(1);
  __syncthreads();
  double lg = 0.0;
  for (int x = 0; x < Lc - 1; ++x) {
    const int cx = dim1[x], cn = dim1[x + 1], Dk = Dk_of(x, d, ring), Dkn = Dk_of(x + 1, d, ring);
    for (int e = threadIdx.x; e < Dkn * cn; e += kThreads) {
      const int kp = e / cn, bb = e % cn, v = kp % d;
      const R* A = env_ptr(w, L, 1, x, v);
      R acc = R(0);
      for (int k = 0; k < Dk; ++k) {
        int kn;
        const R f = hfac(x, k, v, d, ring, psih, &kn);
        if (kn != kp) continue;
        R inner = R(0);
        for (int a = 0; a < cx; ++a) inner += ell[k * cx + a] * A[a * ldE + bb];
        acc += f * inner;
      }
      nxt[e] = acc * phi[x * d + v];
    }
    R loc = R(0);
    for (int e = threadIdx.x; e < Dkn * cn; e += kThreads) loc = fmax(loc, fabs(nxt[e]));
    const R mx = block_max(loc, sm.redr);
    const R inv = mx > R(0) ? R(1) / mx : R(1);
    for (int e = threadIdx.x; e < Dkn * cn; e += kThreads) ell[e] = nxt[e] * inv;
    if (threadIdx.x == 0) lg += mx > R(0) ? log((double)mx) : 0.0;
    __syncthreads();
  }
  const int x = Lc - 1, cx = dim1[x], Dk = Dk_of(x, d, ring);
  R loc = R(0);
  for (int e = threadIdx.x; e < Dk * cx; e += kThreads) {
    const int k = e / cx, a = e % cx;
    for (int v = 0; v < d; ++v) loc += ell[e] * env_ptr(w, L, 1, x, v)[a * ldE] * phi[x * d + v] * hlast(x, k, v, d, ring, psih);
  }
  const R tot = block_sum(loc, sm.redr);
  return lg + log((double)tot);
}

// --------------------------------------------------------- a3/a4: row sampling
// forced != nullptr: evaluate log q of that configuration; else draw with Philox uniforms.
template <typename R>
__device__ double sample_rows(const Group& g, const SliceGeom& s, const PhaseParams& P, Ws<R>& w, SliceSmem<R>& sm,
                              const int8_t* forced, int8_t* out, uint64_t seed, uint32_t step, uint32_t gchain,
                              int* events, int* nonfinite, uint32_t purpose = P_SITE, uint32_t index_base = 0) {
  const WsLayout& L = P.lay;
  const int d = g.d, Lc = s.Lc, ring = s.ring, ldE = L.chimax, Lmax = L.Lmax;
  double logq = 0.0;
  for (int r = 1; r <= s.m; ++r) {
    const R* phi = w.phi + (size_t)(r - 1) * Lmax * d;
    const R* psih = w.psih + (size_t)(r - 1) * Lmax * d * d;
    const R* psiv_up = r >= 2 ? w.psiv + (size_t)(r - 2) * Lmax * d * d : nullptr;
    const int8_t* cfg = forced ? forced : out;
    const int8_t* prev = r >= 2 ? cfg + (size_t)(r - 2) * Lmax : nullptr;
    const int* dimr = w.dims + (size_t)(r - 1) * (Lmax + 1);
    auto ax = [&](int x, int v) -> R {
      R a = phi[x * d + v];
      if (psiv_up) a *= psiv_up[(x * d + prev[x]) * d + v];
      return a;
    };
    auto Rp = [&](int x) { return w.Rv + (size_t)x * L.nmax; };
    // right vectors on the left bond of x = Lc-1 .. 1
    {
      const int x = Lc - 1, cx = dimr[x], Dk = Dk_of(x, d, ring);
      R* Rx = Rp(x);
      for (int e = threadIdx.x; e < Dk * cx; e += kThreads) {
        const int k = e / cx, a = e % cx;
        R acc = R(0);
        for (int v = 0; v < d; ++v) acc += env_ptr(w, L, r, x, v)[a * ldE] * ax(x, v) * hlast(x, k, v, d, ring, psih);
        Rx[e] = acc;
      }
      R loc = R(0);
      for (int e = threadIdx.x; e < Dk * cx; e += kThreads) loc = fmax(loc, fabs(Rx[e]));
      const R mx = block_max(loc, sm.redr);
      const R inv = mx > R(0) ? R(1) / mx : R(1);
      for (int e = threadIdx.x; e < Dk * cx; e += kThreads) Rx[e] *= inv;
      __syncthreads();
    }
    for (int x = Lc - 2; x >= 1; --x) {
      const int cx = dimr[x], cn = dimr[x + 1], Dk = Dk_of(x, d, ring), Dkn = Dk_of(x + 1, d, ring);
      const R* Rn = Rp(x + 1);
      R* t = w.tmp;  // [Dkn][cx]
      for (int e = threadIdx.x; e < Dkn * cx; e += kThreads) {
        const int kp = e / cx, a = e % cx;
        const R* A = env_ptr(w, L, r, x, kp % d) + (size_t)a * ldE;
        R acc = R(0);
        for (int bb = 0; bb < cn; ++bb) acc += A[bb] * Rn[kp * cn + bb];
        t[e] = acc;
      }
      __syncthreads();
      R* Rx = Rp(x);
      R loc = R(0);
      for (int e = threadIdx.x; e < Dk * cx; e += kThreads) {
        const int k = e / cx, a = e % cx;
        R acc = R(0);
        for (int v = 0; v < d; ++v) {
          int kn;
          const R f = hfac(x, k, v, d, ring, psih, &kn);
          acc += ax(x, v) * f * t[kn * cx + a];
        }
        Rx[e] = acc;
        loc = fmax(loc, fabs(acc));
      }
      const R mx = block_max(loc, sm.redr);
      const R inv = mx > R(0) ? R(1) / mx : R(1);
      for (int e = threadIdx.x; e < Dk * cx; e += kThreads) Rx[e] *= inv;
      __syncthreads();
    }
    // left to right
    R* ell = w.tmp + 2 * L.nmax;
    R* ell2 = w.tmp + 3 * L.nmax;
    if (threadIdx.x == 0) ell[0] = R(1);
    __syncthreads();
    int kcur = 0;
    for (int x = 0; x < Lc; ++x) {
      const int cx = dimr[x];
      const bool last = (x == Lc - 1);
      const int cn = last ? 1 : dimr[x + 1];
      double ptv[4];
      for (int v = 0; v < d; ++v) {
        R loc = R(0);
        R fac;
        int kn = 0;
        if (last) fac = hlast(x, kcur, v, d, ring, psih);
        else fac = hfac(x, kcur, v, d, ring, psih, &kn);
        const R* A = env_ptr(w, L, r, x, v);
        const R* Rn = last ? nullptr : Rp(x + 1) + (size_t)kn * cn;
        for (int e = threadIdx.x; e < cx * cn; e += kThreads) {
          const int a = e / cn, bb = e % cn;
          loc += ell[a] * A[(size_t)a * ldE + bb] * (last ? R(1) : Rn[bb]);
        }
        const R tot = block_sum(loc, sm.redr);
        if (threadIdx.x == 0) ptv[v] = (double)tot * (double)fac * (double)ax(x, v);
      }
      if (threadIdx.x == 0) {
        double ssum = 0.0;
        bool bad = false;
        for (int v = 0; v < d; ++v) {
          bad = bad || !isfinite(ptv[v]);        // a NaN or infinite entry makes the conditional unusable
          ssum += ptv[v] > 0.0 ? ptv[v] : 0.0;
        }
        double p[4];
        bool ev = bad || !(ssum > 0.0) || !isfinite(ssum);
        if (ev) {
          for (int v = 0; v < d; ++v) p[v] = 1.0 / d;
          ++*events;
          if (bad || !isfinite(ssum)) ++*nonfinite;
        } else {
          double tt = 0.0;
          for (int v = 0; v < d; ++v) { p[v] = (ptv[v] > 0.0 ? ptv[v] : 0.0) + kFloorEps * ssum; tt += p[v]; }
          for (int v = 0; v < d; ++v) p[v] /= tt;
        }
        int v;
        if (forced) {
          v = forced[(size_t)(r - 1) * Lmax + x];
        } else {
          const double u = philox_uniform(seed, purpose, index_base + (uint32_t)((r - 1) * Lc + x), s.k, s.rax, step,
                                          gchain);
          double cdf = 0.0;
          v = d - 1;
          for (int c = 0; c < d; ++c) {
            cdf += p[c];
            if (u < cdf) { v = c; break; }
          }
        }
        sm.choice = v;
        sm.pt[0] = log(p[v]);
      }
      __syncthreads();
      const int v = sm.choice;
      if (threadIdx.x == 0) logq += sm.pt[0];
      if (threadIdx.x == 0 && !forced) out[(size_t)(r - 1) * Lmax + x] = (int8_t)v;
      if (!last) {
        int kn;
        hfac(x, kcur, v, d, ring, psih, &kn);
        const R* A = env_ptr(w, L, r, x, v);
        R loc = R(0);
        for (int bb = threadIdx.x; bb < cn; bb += kThreads) {
          R acc = R(0);
          for (int a = 0; a < cx; ++a) acc += ell[a] * A[(size_t)a * ldE + bb];
          ell2[bb] = acc;
          loc = fmax(loc, fabs(acc));
        }
        const R mx = block_max(loc, sm.redr);
        const R inv = mx > R(0) ? R(1) / mx : R(1);
        for (int bb = threadIdx.x; bb < cn; bb += kThreads) ell[bb] = ell2[bb] * inv;
        kcur = kn;
        __syncthreads();
      }
    }
    __syncthreads();
  }
  // log q lives in thread 0; broadcast it so that every thread takes the same decision
  if (threadIdx.x == 0) sm.pt[1] = logq;
  __syncthreads();
  logq = sm.pt[1];
  __syncthreads();
  return logq;
}

// ------------------------------------------------------------------ a5: dE, MH
__device__ inline long long delta_energy(const Group& g, const SliceGeom& s, const int8_t* spins, const int32_t* J,
                                         const int8_t* sn, const int8_t* so, int Lmax, long long* red) {
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  long long loc = 0;
  for (int e = threadIdx.x; e < s.m * s.Lc; e += kThreads) {
    const int r = e / s.Lc + 1, x = e % s.Lc;
    const int vn = sn[(r - 1) * Lmax + x], vo = so[(r - 1) * Lmax + x];
    long long h[4];
    site_field(g, s, spins, J, r, x, h);
    loc -= h[vn] - h[vo];
    const int idx = site_index(g, s, r, x);
    if ((x + 1 < s.Lc) || s.ring) {
      const int x2 = (x + 1) % s.Lc;
      loc -= bond_energy(g, s, J, vol, idx, s.ca, vn, sn[(r - 1) * Lmax + x2]) -
             bond_energy(g, s, J, vol, idx, s.ca, vo, so[(r - 1) * Lmax + x2]);
    }
    if (r < s.m) {
      loc -= bond_energy(g, s, J, vol, idx, s.ra, vn, sn[r * Lmax + x]) -
             bond_energy(g, s, J, vol, idx, s.ra, vo, so[r * Lmax + x]);
    }
  }
  return block_sum(loc, red);
}

// n_prop tensor-network proposals from the environments already built for this slice (the E_r
// depend only on the held spins). Proposal j is drawn, its exact energy change against the current
// slice is computed, and Eq. (1) decides; an accepted candidate becomes the current slice with its
// log q. The current slice lives in w.sold (written back at the end), candidates in w.snew.
// Outputs: log q of the original and of the final slice, the number of accepted proposals, and
// E(final) - E(original).
template <typename R>
__device__ void multi_proposal(const Group& g, const SliceGeom& s, const PhaseParams& P, Ws<R>& w, SliceSmem<R>& sm,
                               int8_t* spins, const int32_t* J, double beta, int slice, int axis, uint32_t step,
                               uint32_t gchain, int it, int* events, int* nonfinite) {
  const int Lmax = P.lay.Lmax;
  const int n_sites = s.m * s.Lc;
  const double lq_old = sample_rows<R>(g, s, P, w, sm, w.sold, w.snew, P.seed, step, gchain, events, nonfinite);
  double lq_cur = lq_old;
  long long dE_tot = 0;
  int n_acc = 0;
  for (int j = 0; j < P.n_prop; ++j) {
    const uint32_t pur = j == 0 ? (uint32_t)P_SITE : (uint32_t)P_SITE_K;
    const uint32_t base = j == 0 ? 0u : (uint32_t)((j - 1) * n_sites);
    const double lq_new = sample_rows<R>(g, s, P, w, sm, nullptr, w.snew, P.seed, step, gchain, events, nonfinite,
                                         pur, base);
    const long long dE = delta_energy(g, s, spins, J, w.snew, w.sold, Lmax, sm.redl);
    const double logA = (lq_cur - lq_new) - beta * (double)dE * kJScale;
    const double u = j == 0 ? philox_uniform(P.seed, P_MH, 0, (uint32_t)slice, (uint32_t)s.rax, step, gchain)
                            : philox_uniform(P.seed, P_MH_K, (uint32_t)(j - 1), (uint32_t)slice, (uint32_t)s.rax,
                                             step, gchain);
    const bool finite = isfinite(logA);
    if (!finite && threadIdx.x == 0) ++*nonfinite;
    if (finite && u < exp(fmin(0.0, logA))) {
      for (int e = threadIdx.x; e < n_sites; e += kThreads) {
        const int r = e / s.Lc, x = e % s.Lc;
        w.sold[r * Lmax + x] = w.snew[r * Lmax + x];
      }
      lq_cur = lq_new;
      dE_tot += dE;
      ++n_acc;
      __syncthreads();
    }
  }
  if (n_acc && P.write_back) {
    for (int e = threadIdx.x; e < n_sites; e += kThreads) {
      const int r = e / s.Lc + 1, x = e % s.Lc;
      write_site(g, s, spins, r, x, w.sold[(r - 1) * Lmax + x]);
    }
  }
  if (P.out_spins) {
    for (int e = threadIdx.x; e < Lmax * Lmax; e += kThreads) {
      const int r = e / Lmax, x = e % Lmax;
      P.out_spins[(size_t)it * Lmax * Lmax + e] = (r < s.m && x < s.Lc) ? w.sold[r * Lmax + x] : (int8_t)-1;
    }
  }
  if (threadIdx.x == 0) {
    if (P.out_lq_new) P.out_lq_new[it] = lq_cur;
    if (P.out_lq_old) P.out_lq_old[it] = lq_old;
    if (P.out_acc) P.out_acc[it] = (uint8_t)n_acc;
    if (P.out_dE) P.out_dE[it] = dE_tot;
    if (n_acc && P.acc_counter) atomicAdd(P.acc_counter + gchain, (unsigned int)n_acc);
  }
  __syncthreads();
}

// Work item `it` of a launch: 1 = an update to run, 0 = an unused position (skip), -1 = past the end.
// In a sweep each group owns (slices of the colour class) x chains positions; a group of composite
// layers owns as many as the larger of its two offsets needs (the launch size of a captured graph
// does not depend on t), and the positions beyond this sweep's count are unused.
__device__ inline int find_item(const PhaseParams& P, int it, int& gi, int& chain, int& slice, int& axis,
                                uint32_t& step) {
  if (P.n_items >= 0) {
    gi = P.item_group[it]; chain = P.item_chain[it]; slice = P.item_slice[it];
    axis = P.axis; step = P.step;
    return 1;
  }
  if (P.n_items == -2) {   // every slice normal to P.axis of every chain (cache build)
    axis = P.axis; step = P.step;
    int rem = it;
    for (int g = 0; g < P.n_groups; ++g) {
      const int n = P.groups[g].L[axis], cnt = n * P.groups[g].n_chains;
      if (rem < cnt) { gi = g; chain = rem / n; slice = rem % n; return 1; }
      rem -= cnt;
    }
    return -1;
  }
  const unsigned long long t = *P.sweep_ctr;
  axis = (int)(t % 3ull);
  step = (uint32_t)(t * 4ull + (unsigned long long)P.colour);
  const int offset = (int)((t / 3ull) % 2ull);
  int rem = it;
  for (int g = 0; g < P.n_groups; ++g) {
    const Group& G = P.groups[g];
    const int n = G.L[axis], per = G.bc[axis];
    int nsl, nuse;
    if (G.layers == 2) {
      const int c0 = composite_count(n, per, 0, P.colour), c1 = composite_count(n, per, 1, P.colour);
      nsl = c0 > c1 ? c0 : c1;
      nuse = offset ? c1 : c0;
    } else {
      nsl = nuse = colour_count(n, per, P.colour);
    }
    const int cnt = nsl * G.n_chains;
    if (rem < cnt) {
      gi = g; chain = rem / nsl;
      const int j = rem % nsl;
      if (j >= nuse) return 0;
      slice = G.layers == 2 ? composite_slice(n, per, offset, P.colour, j) : colour_slice(n, per, P.colour, j);
      return 1;
    }
    rem -= cnt;
  }
  return -1;
}

// One kernel instance per GEMM tile (TNMC_GEMM_TILE of the translation unit) and one with the tcgen05
// engine (TNMC_WITH_UMMA), each with its own name.
#if TNMC_WITH_UMMA
#define TNMC_SLICE_KERNEL slice_update_kernel_umma
#elif TNMC_GEMM_TILE == 1
#define TNMC_SLICE_KERNEL slice_update_kernel_t32
#elif TNMC_GEMM_TILE == 2
#define TNMC_SLICE_KERNEL slice_update_kernel_t128
#else
#define TNMC_SLICE_KERNEL slice_update_kernel
#endif

template <typename R>
__global__ void __launch_bounds__(kThreads, 2) TNMC_SLICE_KERNEL(PhaseParams P, int total_items) {
  __shared__ SliceSmem<R> sm;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Ws<R> w = bind_ws<R>(P);
  if (P.eig_smem) w.dyn = reinterpret_cast<R*>(dyn_smem);
  w.stage = nullptr;
  if (P.umma_stage) {   // 128-byte aligned start inside the dynamic region (the host reserves the slack)
    const uintptr_t a = reinterpret_cast<uintptr_t>(dyn_smem);
    w.stage = dyn_smem + ((128 - (a & 127)) & 127);
  }
  int events = 0, nonfinite = 0;
  R* const E_ws = w.E;
  int* const dims_ws = w.dims;
  for (int it = blockIdx.x; it < total_items; it += gridDim.x) {
    int gi, chain, slice, axis;
    uint32_t step;
    const int found = find_item(P, it, gi, chain, slice, axis, step);
    if (found < 0) break;
    if (found == 0) continue;
    const Group& g = P.groups[gi];
    const uint32_t gchain = (uint32_t)(g.chain_base + chain);
    int proposal = P.proposal;
    if (P.n_items < 0 && P.net_every > 0) {
      const unsigned long long t = *P.proposal_ctr;
      proposal = (t % (unsigned long long)P.net_every) == (unsigned long long)(P.net_every - 1) ? 1 : 0;
    }
    // environments of a cached item live in its slot: contracted there (build) or read from there (use);
    // only tensor-network proposals use the cache
    w.E = E_ws;
    w.dims = dims_ws;
    bool cached = false;
    int* meta = nullptr;
    if (P.cache_mode != CACHE_OFF && proposal == 0) {
      char* slot = P.cache + (((size_t)gchain * 3 + axis) * P.cache_lmax + slice) * P.cache_stride;
      meta = reinterpret_cast<int*>(slot + P.cache_meta_off);
      if (P.cache_mode == CACHE_USE) {
        cached = meta[2] == 1;
      } else if (P.cache_mode == CACHE_SWEEP) {
        const unsigned long long t = *P.sweep_ctr, k = (unsigned long long)P.cache_every;
        cached = meta[2] == 1 && !(k > 0 && t % k == k - 1);
      }
      if (cached || P.cache_mode == CACHE_BUILD) {
        w.E = reinterpret_cast<R*>(slot);
        w.dims = reinterpret_cast<int*>(slot + P.cache_dims_off);
      }
    }
    const SliceGeom s = cached ? geom_with_lines(g, axis, slice, meta[0], meta[1])
                               : make_geom(g, axis, slice, P.seed, step, gchain);
    const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
    int8_t* spins = g.spins + (size_t)chain * vol;
    const int32_t* J = g.J + (size_t)g.inst[chain] * 3 * vol;
    const double beta = g.beta[chain];
    const int Lmax = P.lay.Lmax;
    build_weights<R>(g, s, spins, J, beta * P.env_beta_factor, P, w, sm);
    if (!cached) {   // E_m = 1
      for (int e = threadIdx.x; e <= s.Lc; e += kThreads) w.dims[(size_t)(s.m - 1) * (Lmax + 1) + e] = 1;
      for (int e = threadIdx.x; e < s.Lc * g.d; e += kThreads) *env_ptr(w, P.lay, s.m, e / g.d, e % g.d) = R(1);
    }
    __syncthreads();
    double lq_new, lq_old;
    if (proposal == 1) {
      // learned proposal: conditioning, raster-order draw, teacher-forced log q of the current slice
      const int Pm = P.net_Pmax, Pn = s.m * s.Lc;
      float* nws = P.net_ws + (size_t)blockIdx.x * P.net_ws_stride;
      float* cond = nws;
      float* zb = cond + (size_t)P.net.Cc * Pm;
      float* xb = zb + (size_t)P.net.NL * P.net.H * Pm;
      int8_t* sc = reinterpret_cast<int8_t*>(xb + (size_t)P.net.NL * P.net.H * Pm);
      int8_t* oc = sc + Pm;
      net_cond(g, s, spins, J, beta, cond, Pm);
      lq_new = net_sample(P.net, P.net_W, cond, sc, s.m, s.Lc, xb, zb, Pm, P.seed, (uint32_t)slice, (uint32_t)axis,
                          step, gchain, sm.redd, &sm.choice);
      for (int e = threadIdx.x; e < Pn; e += kThreads) {
        const int r = e / s.Lc, x = e % s.Lc;
        w.snew[r * Lmax + x] = sc[e];
        oc[e] = w.sold[r * Lmax + x];
      }
      __syncthreads();
      net_forward(P.net, P.net_W, cond, oc, s.m, s.Lc, zb, xb, Pm);
      lq_old = net_logq(P.net, xb + (size_t)(P.net.NL - 1) * P.net.H * Pm, oc, Pn, Pm, sm.redd);
    } else {
      double lognorm = 0.0;
      if (!cached)
        for (int r = s.m; r >= 2; --r)
          lognorm += P.route == ROUTE_DM ? env_step_dm<R>(g, s, r, P, w, sm) : env_step_lq<R>(g, s, r, P, w, sm);
      if (P.cache_mode == CACHE_BUILD) {
        if (threadIdx.x == 0) { meta[0] = s.y0; meta[1] = s.x0; meta[2] = 1; }
        __syncthreads();
        continue;
      }
      if (P.logz_only) {
        const double lz = close_row1<R>(g, s, P, w, sm);
        const double tot = lz + lognorm + sm.lscale;
        if (threadIdx.x == 0) {
          P.out_logz[it] = tot;
          if (!isfinite(tot)) ++nonfinite;
        }
        __syncthreads();
        continue;
      }
      TNMC_PROF_BEGIN(3);
      if (P.n_prop > 1) {
        // several proposals from this environment build, as an independence-sampler chain on the slice
        multi_proposal<R>(g, s, P, w, sm, spins, J, beta, slice, axis, step, gchain, it, &events, &nonfinite);
        TNMC_PROF_END(3);
        continue;
      }
      lq_new = sample_rows<R>(g, s, P, w, sm, nullptr, w.snew, P.seed, step, gchain, &events, &nonfinite);
      lq_old = sample_rows<R>(g, s, P, w, sm, w.sold, w.snew + 0, P.seed, step, gchain, &events, &nonfinite);
      TNMC_PROF_END(3);
    }
    const long long dE = delta_energy(g, s, spins, J, w.snew, w.sold, Lmax, sm.redl);
    const double logA = (lq_old - lq_new) - beta * (double)dE * kJScale;
    const double u = philox_uniform(P.seed, P_MH, 0, (uint32_t)slice, (uint32_t)s.rax, step, gchain);
    // a non-finite log ratio (it cannot arise from finite inputs) rejects the move and is latched
    const bool finite = isfinite(logA);
    if (!finite && threadIdx.x == 0) ++nonfinite;
    const bool acc = finite && u < exp(fmin(0.0, logA));
    if (acc && P.write_back) {
      for (int e = threadIdx.x; e < s.m * s.Lc; e += kThreads) {
        const int r = e / s.Lc + 1, x = e % s.Lc;
        write_site(g, s, spins, r, x, w.snew[(r - 1) * Lmax + x]);
      }
    }
    if (acc && P.record && proposal == 0 && P.rb_slots > 0) {
      // item it of this launch owns slot (positions offered before the launch + it) mod slots, so the
      // buffer's contents do not depend on the order in which CTAs finish; a rejected item leaves its
      // slot as it was
      const size_t slot = (size_t)((*P.rb_counter + (unsigned long long)it) % (unsigned long long)P.rb_slots);
      const int Pm = P.net_Pmax;
      net_cond(g, s, spins, J, beta, P.rb_cond + slot * (size_t)P.net.Cc * Pm, Pm);
      for (int e = threadIdx.x; e < s.m * s.Lc; e += kThreads)
        P.rb_spins[slot * Pm + e] = w.snew[(e / s.Lc) * Lmax + e % s.Lc];
      if (threadIdx.x == 0) { P.rb_meta[2 * slot] = s.m; P.rb_meta[2 * slot + 1] = s.Lc; }
      __syncthreads();
    }
    if (P.out_spins) {
      for (int e = threadIdx.x; e < Lmax * Lmax; e += kThreads) {
        const int r = e / Lmax, x = e % Lmax;
        P.out_spins[(size_t)it * Lmax * Lmax + e] = (r < s.m && x < s.Lc) ? w.snew[r * Lmax + x] : (int8_t)-1;
      }
    }
    if (threadIdx.x == 0) {
      if (P.out_lq_new) P.out_lq_new[it] = lq_new;
      if (P.out_lq_old) P.out_lq_old[it] = lq_old;
      if (P.out_acc) P.out_acc[it] = acc ? 1 : 0;
      if (P.out_dE) P.out_dE[it] = dE;
      if (acc && P.acc_counter) atomicAdd(P.acc_counter + gchain, 1u);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && events && P.event_counter) atomicAdd(P.event_counter, (unsigned long long)events);
  if (threadIdx.x == 0 && nonfinite && P.status) atomicOr(P.status, (unsigned int)ST_NONFINITE);
}

}  // namespace tnmc
