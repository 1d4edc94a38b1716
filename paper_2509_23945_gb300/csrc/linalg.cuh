// CTA-cooperative dense linear algebra on small matrices: tiled GEMM, a blocked
// Householder LQ factorisation, one-sided (Hestenes) Jacobi orthogonalisation
// and a cyclic Jacobi eigensolver for symmetric matrices. Every routine is
// called by all threads of the CTA and ends with a barrier.
#pragma once

#include "common.cuh"

namespace tnmc {

// K-chunk of the CUDA-core GEMM (16: the prefetch registers fit without spills).
template <typename R> struct GemmKC { static constexpr int v = 16; };

// Output tile of the CUDA-core GEMM, fixed per translation unit: TNMC_GEMM_TILE 0 (default) 64 x 64,
// 1: 32 x 32, 2: 128 x 64 (rows x columns). The slice kernel is compiled once per tile in its own
// translation unit (kernel names differ) and the tuning picks one at run time. Every output element
// accumulates its K products in the same order whatever the tile, so the tile never changes a result.
#ifndef TNMC_GEMM_TILE
#define TNMC_GEMM_TILE 0
#endif
#if TNMC_GEMM_TILE == 1
constexpr int kGemmTM = 32, kGemmTN = 32;
#elif TNMC_GEMM_TILE == 2
constexpr int kGemmTM = 128, kGemmTN = 64;
#else
constexpr int kGemmTM = 64, kGemmTN = 64;
#endif

template <typename R>
struct __align__(16) GemmSmem {
  R a[GemmKC<R>::v][kGemmTM + 4];
  R b[GemmKC<R>::v][kGemmTN + 4];
};

// C[M x N] = alpha * op(A) * op(B) + beta * C, row-major with leading dims.
// op(A)[i][k] = ta ? A[k*lda + i] : A[i*lda + k]; op(B)[k][j] = tb ? B[j*ldb + k] : B[k*ldb + j].
// beta == 0 never reads C. Thread (ty, tx) of a 16x16 grid owns rows RM ty + i and columns
// RN tx + j of each TM x TN output tile (RM = TM / 16, RN = TN / 16), so each k step reads its
// RM A and RN B values with 16-byte (or 8-byte) shared-memory loads. The next K-chunk is loaded
// into registers while the current one is multiplied out of shared memory, so global (L2 / HBM)
// latency overlaps the arithmetic.
// Consecutive shared-memory values (16-byte aligned for 4, 8-byte for 2) into registers.
template <typename Acc>
__device__ inline void load4(const float* p, Acc* v) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = (Acc)x.x; v[1] = (Acc)x.y; v[2] = (Acc)x.z; v[3] = (Acc)x.w;
}
template <typename Acc>
__device__ inline void load4(const double* p, Acc* v) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  const double2 y = *reinterpret_cast<const double2*>(p + 2);
  v[0] = (Acc)x.x; v[1] = (Acc)x.y; v[2] = (Acc)y.x; v[3] = (Acc)y.y;
}
template <typename Acc>
__device__ inline void load2(const float* p, Acc* v) {
  const float2 x = *reinterpret_cast<const float2*>(p);
  v[0] = (Acc)x.x; v[1] = (Acc)x.y;
}
template <typename Acc>
__device__ inline void load2(const double* p, Acc* v) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  v[0] = (Acc)x.x; v[1] = (Acc)x.y;
}
template <int N, typename R, typename Acc>
__device__ inline void load_row(const R* p, Acc* v) {
  if constexpr (N == 2) {
    load2(p, v);
  } else {
#pragma unroll
    for (int q = 0; q < N; q += 4) load4(p + q, v + q);
  }
}

// b_lower: op(B) is lower triangular (op(B)[k][j] = 0 for k < j), so the output tile of columns
// n0.. skips the K range below n0. The skipped terms are exact zeros, so results are unchanged.
template <typename R, typename Acc = R>
__device__ void cta_gemm(int M, int N, int K, R alpha, const R* A, int lda, bool ta, const R* B, int ldb,
                         bool tb, R beta, R* C, int ldc, GemmSmem<R>& sm, bool b_lower = false) {
  constexpr int KC = GemmKC<R>::v;
  constexpr int TM = kGemmTM, TN = kGemmTN, RM = TM / 16, RN = TN / 16;
  constexpr int PA = KC * TM / kThreads;   // elements of each operand a thread stages per chunk
  constexpr int PB = KC * TN / kThreads;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  R ra[PA], rb[PB];
  constexpr int PMAX = PA > PB ? PA : PB;
  auto fetch = [&](int m0, int n0, int k0) {
#pragma unroll
    for (int t = 0; t < PMAX; ++t) {
      const int e = tid + t * kThreads;
      if (t < PA) {
        int kk, mm;
        if (ta) { kk = e / TM; mm = e % TM; } else { mm = e / KC; kk = e % KC; }
        const int gm = m0 + mm, gk = k0 + kk;
        ra[t] = (gm < M && gk < K) ? (ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : R(0);
      }
      if (t < PB) {
        int kb, nb;
        if (tb) { nb = e / KC; kb = e % KC; } else { kb = e / TN; nb = e % TN; }
        const int gn = n0 + nb, gkb = k0 + kb;
        rb[t] = (gn < N && gkb < K) ? (tb ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn]) : R(0);
      }
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int t = 0; t < PMAX; ++t) {
      const int e = tid + t * kThreads;
      if (t < PA) {
        int kk, mm;
        if (ta) { kk = e / TM; mm = e % TM; } else { mm = e / KC; kk = e % KC; }
        sm.a[kk][mm] = ra[t];
      }
      if (t < PB) {
        int kb, nb;
        if (tb) { nb = e / KC; kb = e % KC; } else { kb = e / TN; nb = e % TN; }
        sm.b[kb][nb] = rb[t];
      }
    }
  };
  for (int m0 = 0; m0 < M; m0 += TM) {
    for (int n0 = 0; n0 < N; n0 += TN) {
      Acc acc[RM][RN];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = Acc(0);
      const int kb0 = b_lower ? (n0 / KC) * KC : 0;
      if (K > kb0) fetch(m0, n0, kb0);
      for (int k0 = kb0; k0 < K; k0 += KC) {
        stash();
        __syncthreads();
        if (k0 + KC < K) fetch(m0, n0, k0 + KC);   // in flight while this chunk is multiplied
        const int kend = (K - k0) < KC ? (K - k0) : KC;
        for (int kk = 0; kk < kend; ++kk) {
          Acc av[RM], bv[RN];
          load_row<RM>(&sm.a[kk][RM * ty], av);
          load_row<RN>(&sm.b[kk][RN * tx], bv);
#pragma unroll
          for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
      }
      // epilogue: with beta != 0 every C value is loaded before any store, so the loads are in
      // flight together instead of one global round trip per element
      R cold[RM][RN];
      if (beta != R(0)) {
#pragma unroll
        for (int i = 0; i < RM; ++i) {
          const int gm = m0 + RM * ty + i;
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            const int gn = n0 + RN * tx + j;
            cold[i][j] = (gm < M && gn < N) ? C[(size_t)gm * ldc + gn] : R(0);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RM; ++i) {
        const int gm = m0 + RM * ty + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          const int gn = n0 + RN * tx + j;
          if (gn >= N) continue;
          const R v = alpha * (R)acc[i][j];
          C[(size_t)gm * ldc + gn] = (beta == R(0)) ? v : v + beta * cold[i][j];
        }
      }
    }
  }
  __syncthreads();
}

template <typename R> struct Eps;
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct Eps<float> { static constexpr float v = 1.1920929e-07f; };

// Rotation list of one Jacobi round, kept in the working precision (no
// float <-> double conversions in the FP32 path: GB300 runs them on its FP64 pipe).
template <typename R>
struct JacobiSmem {
  int p[128];
  int q[128];
  R c[128];
  R s[128];
  int flag;
};

// Cyclic Jacobi eigensolver for a symmetric n x n matrix (n <= 256). Rotations
// follow the symmetric 2x2 Schur decomposition of Golub & Van Loan (sym.schur2);
// pairs are scheduled with the round-robin (circle) ordering so each round's
// rotations act on disjoint index pairs. A (lda, padded to avoid bank
// conflicts) is symmetric; VT receives the eigenvectors as rows (VT[k][row] =
// component `row` of eigenvector k, leading dimension ldv), so the per-round
// update of two eigenvectors touches contiguous memory. Same rotations and
// each round applies J_i^T A[blk i, blk j] J_j
// to the 2x2 blocks of every pair of index pairs at once (pairs are disjoint,
// so blocks do not overlap); only the upper triangle of blocks is computed and
// mirrored: one barrier per round. A rotation is significant when
// |a_pq| > tol sqrt(|a_pp a_qq|) + eps * max|a_ii|; the absolute term stops
// rotations of entries that are already at the rounding level of A.
template <typename R>
__device__ int cta_jacobi_eig_fused(int n, R* A, int lda, R* VT, int ldv, int max_sweeps, JacobiSmem<R>& js,
                                    R* red, int floor_mode) {
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += kThreads) {
    const int i = e / n, j = e % n;
    VT[(size_t)i * ldv + j] = (i == j) ? R(1) : R(0);
  }
  R loc = R(0);
  for (int i = tid; i < n; i += kThreads) loc = fmax(loc, fabs(A[(size_t)i * lda + i]));
  const R scale = block_max(loc, red);
  if (n <= 1) return 0;
  const int ne = n + (n & 1);
  const int np = ne / 2;
  const R tol = R(4) * Eps<R>::v;
  // absolute floor: 0 none, 1 eps^2 n max|a_ii|, 2 eps max|a_ii|
  const R floor_abs = floor_mode == 0 ? R(0)
                    : floor_mode == 1 ? Eps<R>::v * Eps<R>::v * (R)n * scale : Eps<R>::v * scale;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    ++sweeps;
    if (tid == 0) js.flag = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      for (int i = tid; i < np; i += kThreads) {
        const int a = (i == 0) ? 0 : ((round + i - 1) % (ne - 1)) + 1;
        const int b = ((round + ne - 1 - i - 1) % (ne - 1)) + 1;
        const int p = a < b ? a : b, q = a < b ? b : a;
        R c = R(1), s = R(0);
        if (q < n) {
          const R apq = A[(size_t)p * lda + q];
          const R app = A[(size_t)p * lda + p];
          const R aqq = A[(size_t)q * lda + q];
          const R thr = tol * sqrt(fabs(app * aqq)) + floor_abs;
          if (fabs(apq) > thr) {
            js.flag = 1;
            const R tau = (aqq - app) / (R(2) * apq);
            const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
            const R cc = R(1) / sqrt(R(1) + t * t);
            c = cc;
            s = t * cc;
          }
        }
        js.p[i] = p;
        js.q[i] = q;
        js.c[i] = c;
        js.s[i] = s;
      }
      __syncthreads();
      // threads as an 8 x 32 grid: ti walks block rows, tj block columns / vector rows
      const int tj = tid & 31, ti = tid >> 5;
      for (int i = ti; i < np; i += kThreads / 32) {
        const R si = js.s[i];
        const R ci = js.c[i];
        const int pi = js.p[i], qi = js.q[i];
        const bool hq_i = qi < n;
        for (int j = i + tj; j < np; j += 32) {
          const R sj = js.s[j];
          if (si == R(0) && sj == R(0)) continue;
          const R cj = js.c[j];
          const int pj = js.p[j], qj = js.q[j];
          const bool hq_j = qj < n;
          const R b00 = A[(size_t)pi * lda + pj];
          const R b01 = hq_j ? A[(size_t)pi * lda + qj] : R(0);
          const R b10 = hq_i ? A[(size_t)qi * lda + pj] : R(0);
          const R b11 = (hq_i && hq_j) ? A[(size_t)qi * lda + qj] : R(0);
          const R t00 = cj * b00 - sj * b01, t01 = sj * b00 + cj * b01;
          const R t10 = cj * b10 - sj * b11, t11 = sj * b10 + cj * b11;
          R n00 = ci * t00 - si * t10, n01 = ci * t01 - si * t11;
          R n10 = si * t00 + ci * t10, n11 = si * t01 + ci * t11;
          if (i == j) { n01 = R(0); n10 = R(0); }
          A[(size_t)pi * lda + pj] = n00;
          A[(size_t)pj * lda + pi] = n00;
          if (hq_j) { A[(size_t)pi * lda + qj] = n01; A[(size_t)qj * lda + pi] = n01; }
          if (hq_i) { A[(size_t)qi * lda + pj] = n10; A[(size_t)pj * lda + qi] = n10; }
          if (hq_i && hq_j) { A[(size_t)qi * lda + qj] = n11; A[(size_t)qj * lda + qi] = n11; }
        }
        // eigenvector rows p_i, q_i of VT (contiguous in `row`); FP32 rows are 16-byte aligned
        // when ldv % 4 == 0, so four components move per load
        if (si != R(0)) {
          R* vp = VT + (size_t)pi * ldv;
          R* vq = VT + (size_t)qi * ldv;
          int row0 = 0;
          if constexpr (sizeof(R) == 4) {
            if ((ldv & 3) == 0) {
              row0 = n & ~3;
              for (int row = tj * 4; row < row0; row += 128) {
                float4 x = *reinterpret_cast<const float4*>(vp + row);
                float4 y = *reinterpret_cast<const float4*>(vq + row);
                float4 a, b;
                a.x = ci * x.x - si * y.x; b.x = si * x.x + ci * y.x;
                a.y = ci * x.y - si * y.y; b.y = si * x.y + ci * y.y;
                a.z = ci * x.z - si * y.z; b.z = si * x.z + ci * y.z;
                a.w = ci * x.w - si * y.w; b.w = si * x.w + ci * y.w;
                *reinterpret_cast<float4*>(vp + row) = a;
                *reinterpret_cast<float4*>(vq + row) = b;
              }
            }
          }
          for (int row = row0 + tj; row < n; row += 32) {
            const R vx = vp[row], vy = vq[row];
            vp[row] = ci * vx - si * vy;
            vq[row] = si * vx + ci * vy;
          }
        }
      }
      __syncthreads();
    }
    const int f = js.flag;
    __syncthreads();
    if (!f) break;
  }
  return sweeps;
}

// rank[i] = position of eigenvalue i in descending order (ties by index).
template <typename R>
__device__ void cta_rank_desc(int n, const R* A, int lda, int* rank) {
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const R wi = A[(size_t)i * lda + i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const R wj = A[(size_t)j * lda + j];
      r += (wj > wi) || (wj == wi && j < i);
    }
    rank[i] = r;
  }
  __syncthreads();
}

// ------------------------------------------------------------- Householder LQ
// Reflector data of one panel: tau_i and the triangular factor T of the compact
// WY form H_0 H_1 ... H_{b-1} = I - V T V^T (Schreiber & Van Loan, 1989).
template <typename R>
struct LqSmem {
  R T[32][33];
  R S[32][33];   // V^T V of the panel
  R tau[32];
};

// Panel height of cta_lq (fixed, so the arithmetic does not depend on where the panel is staged).
constexpr int kLqPanel = 32;

// Row helpers of the LQ panel, one warp per row, over columns [c0, mm) of rows with leading
// dimension ldp. For float rows with ldp a multiple of 4 the body moves float4 vectors (a scalar
// head reaches the first aligned column); the sums are reduced over the warp.
template <typename R>
__device__ inline R row_dot(const R* a, const R* b, int c0, int mm, int ldp, int lane) {
  R acc = R(0);
  int cb = c0;
  if constexpr (sizeof(R) == 4) {
    if ((ldp & 3) == 0) {
      cb = (c0 + 3) & ~3;
      if (cb > mm) cb = mm;
      if (c0 + lane < cb) acc += a[c0 + lane] * b[c0 + lane];
      for (int c = cb + 4 * lane; c + 3 < mm; c += 128) {
        const float4 x = *reinterpret_cast<const float4*>(a + c);
        const float4 y = *reinterpret_cast<const float4*>(b + c);
        acc += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
      }
      return warp_sum(acc);
    }
  }
  for (int c = c0 + lane; c < mm; c += 32) acc += a[c] * b[c];
  return warp_sum(acc);
}

// a[c] += f * b[c] over [c0, mm)
template <typename R>
__device__ inline void row_axpy(R* a, const R* b, R f, int c0, int mm, int ldp, int lane) {
  if constexpr (sizeof(R) == 4) {
    if ((ldp & 3) == 0) {
      int cb = (c0 + 3) & ~3;
      if (cb > mm) cb = mm;
      if (c0 + lane < cb) a[c0 + lane] += f * b[c0 + lane];
      for (int c = cb + 4 * lane; c + 3 < mm; c += 128) {
        float4 x = *reinterpret_cast<float4*>(a + c);
        const float4 y = *reinterpret_cast<const float4*>(b + c);
        x.x += f * y.x; x.y += f * y.y; x.z += f * y.z; x.w += f * y.w;
        *reinterpret_cast<float4*>(a + c) = x;
      }
      return;
    }
  }
  for (int c = c0 + lane; c < mm; c += 32) a[c] += f * b[c];
}

// In-place LQ factorisation A = L Q of the row-major n x m matrix A (leading
// dimension lda) by Householder reflectors applied from the right (Golub & Van
// Loan, Sec. 5.2, transposed). On return A[i][j] holds L for j <= i and
// j < min(n, m) and 0 right of the diagonal; Q is not formed (the callers need
// only L, whose Gram matrix L L^T equals A A^T without forming it).
//
// Rows are processed in panels of kLqPanel rows staged in `pan` (room for
// kLqPanel x m elements; shared memory when it fits). Inside
// a panel, row r belongs to warp r % 8: the owner of row i builds reflector i
// from its row (v_i = [1, x_{i+1..}/(alpha - beta)], tau_i = (beta - alpha)/beta,
// beta = -sign(alpha) |x|), and after one barrier every warp applies it to its
// own rows below, so a panel costs one CTA barrier per reflector. The panel's
// reflectors are then accumulated into T and applied to the rows below the
// panel as A_t <- A_t - ((A_t V) T) V^T: three GEMMs. Wb and Wb2 hold
// (n x 32) elements each, Sb 32 x 32.
//
// Staircase (rpb > 0): row r is zero beyond column ext(r) = min(m, (r / rpb + 1) * estep), with ext
// nondecreasing in r. A panel's reflectors then live in columns below the extent of its last row,
// so the panel and its trailing update stop there; the skipped entries are exact zeros, and the
// result is bitwise that of the dense factorisation.
template <typename R>
__device__ void cta_lq(int n, int m, R* A, int lda, R* pan, R* Wb, R* Wb2, R* Sb, LqSmem<R>& ls, GemmSmem<R>& gs,
                       int rpb = 0, int estep = 0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kmax = n < m ? n : m;
  const int ib = kLqPanel;
  for (int i0 = 0; i0 < kmax; i0 += ib) {
    const int nb = (kmax - i0) < ib ? (kmax - i0) : ib;
    int mext = m;
    if (rpb > 0) {
      int e = ((i0 + nb - 1) / rpb + 1) * estep;
      if (e < i0 + nb) e = i0 + nb;   // the panel always covers its own diagonal
      mext = e < m ? e : m;
    }
    const int mm = mext - i0;
    const int ldp = mm;
    TNMC_PROF_BEGIN(12);
    for (int e = tid; e < nb * mm; e += kThreads) {
      const int r = e / mm, c = e - r * mm;
      pan[(size_t)r * ldp + c] = A[(size_t)(i0 + r) * lda + i0 + c];
    }
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
      __syncwarp();
      if (warp == i % kWarps) {
        R* row = pan + (size_t)i * ldp;
        const R ss = row_dot(row, row, i + 1, mm, ldp, lane);
        const R alpha = row[i];
        R tau = R(0), beta = alpha;
        if (ss > R(0)) {
          const R nrm = sqrt(alpha * alpha + ss);
          beta = alpha >= R(0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          const R scal = R(1) / (alpha - beta);
          for (int c = i + 1 + lane; c < mm; c += 32) row[c] *= scal;
        }
        __syncwarp();
        if (lane == 0) { row[i] = beta; ls.tau[i] = tau; }
      }
      __syncthreads();
      const R tau = ls.tau[i];
      if (tau != R(0)) {
        const R* v = pan + (size_t)i * ldp;
        for (int r = i + 1; r < nb; ++r) {
          if (r % kWarps != warp) continue;
          R* row = pan + (size_t)r * ldp;
          const R sdot = row_dot(row, v, i + 1, mm, ldp, lane);
          const R f = tau * (row[i] + sdot);
          __syncwarp();
          if (lane == 0) row[i] -= f;
          row_axpy(row, v, -f, i + 1, mm, ldp, lane);
        }
      }
    }
    __syncthreads();
    // L part of the panel rows back to A (zeros right of the diagonal); the panel becomes V^T
    for (int e = tid; e < nb * mm; e += kThreads) {
      const int r = e / mm, c = e - r * mm;
      const R val = pan[(size_t)r * ldp + c];
      A[(size_t)(i0 + r) * lda + i0 + c] = c <= r ? val : R(0);
    }
    __syncthreads();
    TNMC_PROF_END(12);
    const int nt = n - i0 - nb;
    if (nt <= 0) continue;
    TNMC_PROF_BEGIN(13);
    for (int e = tid; e < nb * mm; e += kThreads) {
      const int r = e / mm, c = e - r * mm;
      if (c < r) pan[(size_t)r * ldp + c] = R(0);
      else if (c == r) pan[(size_t)r * ldp + c] = R(1);
    }
    __syncthreads();
    // S = V^T V (only the strict upper triangle is used)
    cta_gemm<R>(nb, nb, mm, R(1), pan, ldp, false, pan, ldp, true, R(0), &ls.S[0][0], 33, gs);
    // T (forward, columnwise): T[b][b] = tau_b, T[0:b, b] = -tau_b T[0:b, 0:b] S[0:b, b]. Lane a owns row a.
    if (warp == 0) {
      const int a = lane;
      for (int b = 0; b < nb; ++b) {
        R val = R(0);
        if (a < b) {
          R acc = R(0);
          for (int c = a; c < b; ++c) acc += ls.T[a][c] * ls.S[c][b];
          val = -ls.tau[b] * acc;
        } else if (a == b) {
          val = ls.tau[b];
        }
        if (a < nb) ls.T[a][b] = val;
      }
    }
    __syncthreads();
    TNMC_PROF_END(13);
    TNMC_PROF_BEGIN(14);
    R* At = A + (size_t)(i0 + nb) * lda + i0;
    cta_gemm<R>(nt, nb, mm, R(1), At, lda, false, pan, ldp, true, R(0), Wb, nb, gs);            // W = A_t V
    cta_gemm<R>(nt, nb, nb, R(1), Wb, nb, false, &ls.T[0][0], 33, false, R(0), Wb2, nb, gs);    // W T
    cta_gemm<R>(nt, mm, nb, R(-1), Wb2, nb, false, pan, ldp, false, R(1), At, lda, gs);         // A_t -= W T V^T
    TNMC_PROF_END(14);
  }
  __syncthreads();
}

// ------------------------------------------------ one-sided Jacobi (Hestenes)
// Orthogonalises the k rows of Z (each of length n, leading dimension ldz) by
// plane rotations of row pairs (Hestenes, 1958; the one-sided Jacobi SVD of
// Demmel & Veselic, 1992). For a pair (p, q) with alpha = |z_p|^2,
// beta = |z_q|^2 and gamma = z_p . z_q, a rotation is taken when
// |gamma| > tol sqrt(alpha beta), with zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t,
// z_p <- c z_p - s z_q, z_q <- s z_p + c z_q, which makes the pair orthogonal.
// If Z^T = X V then X = U S W^T has U = the normalised rows of the result and S
// their norms: the singular values and left singular vectors of X are found
// from X itself, never from X X^T, so small singular values keep their
// relative accuracy. Pairs are scheduled in round-robin order (each round
// rotates disjoint pairs, g threads per pair); one barrier per round.
// Rows below a floor relative to the largest are not rotated (see floor_rel).
// t is formed without squaring zeta when |zeta| > 1, so it cannot overflow. On return nrm2[j] = |z_j|^2 and
// *max_nrm2 = max_j nrm2[j]. Returns the number of sweeps.
// One pair of rows (p, q) of the one-sided Jacobi, held in registers by the g threads of its group:
// thread `sub` owns elements sub*V + t*g*V + [0, V) (V = 4 for float rows whose length and leading
// dimension are multiples of 4, read as float4; else V = 1). Computes the three inner products,
// reduces them over the group and applies the rotation. NV vectors per thread cover the row.
template <typename R, int V, int NV>
__device__ inline void jacobi_pair(R* zp, R* zq, int n, int sub, int g, bool active, R tol, R floor2, int* flag) {
  R x[NV * V], y[NV * V];
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const int e = (sub + t * g) * V;
    if (active && e < n) {
      if constexpr (V == 4) {
        const float4 a = *reinterpret_cast<const float4*>(zp + e);
        const float4 b = *reinterpret_cast<const float4*>(zq + e);
        x[4 * t] = a.x; x[4 * t + 1] = a.y; x[4 * t + 2] = a.z; x[4 * t + 3] = a.w;
        y[4 * t] = b.x; y[4 * t + 1] = b.y; y[4 * t + 2] = b.z; y[4 * t + 3] = b.w;
      } else {
        x[t] = zp[e];
        y[t] = zq[e];
      }
    } else {
#pragma unroll
      for (int i = 0; i < V; ++i) { x[V * t + i] = R(0); y[V * t + i] = R(0); }
    }
  }
  R al = R(0), be = R(0), ga = R(0);
#pragma unroll
  for (int i = 0; i < NV * V; ++i) {
    al += x[i] * x[i];
    be += y[i] * y[i];
    ga += x[i] * y[i];
  }
  for (int o = g >> 1; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (active && al > floor2 && be > floor2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
    const R zeta = (be - al) / (R(2) * ga);
    const R az = fabs(zeta);
    const R den = az > R(1) ? az * (R(1) + sqrt(R(1) + (R(1) / az) * (R(1) / az))) : az + sqrt(R(1) + az * az);
    const R t = (zeta >= R(0) ? R(1) : R(-1)) / den;
    const R c = R(1) / sqrt(R(1) + t * t);
    const R s = c * t;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int e = (sub + u * g) * V;
      if (e < n) {
        if constexpr (V == 4) {
          float4 a, b;
          a.x = c * x[4 * u] - s * y[4 * u];         b.x = s * x[4 * u] + c * y[4 * u];
          a.y = c * x[4 * u + 1] - s * y[4 * u + 1]; b.y = s * x[4 * u + 1] + c * y[4 * u + 1];
          a.z = c * x[4 * u + 2] - s * y[4 * u + 2]; b.z = s * x[4 * u + 2] + c * y[4 * u + 2];
          a.w = c * x[4 * u + 3] - s * y[4 * u + 3]; b.w = s * x[4 * u + 3] + c * y[4 * u + 3];
          *reinterpret_cast<float4*>(zp + e) = a;
          *reinterpret_cast<float4*>(zq + e) = b;
        } else {
          zp[e] = c * x[u] - s * y[u];
          zq[e] = s * x[u] + c * y[u];
        }
      }
    }
    if (sub == 0) *flag = 1;
  }
}

// The rows held by one group's registers when n <= NV * V * g.
template <typename R, int V, int NV>
__device__ inline int jacobi_sweeps(int k, int n, R* Z, int ldz, int max_sweeps, R tol, R floor2, int* flag_sh) {
  const int tid = threadIdx.x;
  const int ne = k + (k & 1), np = ne / 2;
  int g = kThreads / np;
  g = g >= 32 ? 32 : (g >= 16 ? 16 : (g >= 8 ? 8 : (g >= 4 ? 4 : (g >= 2 ? 2 : 1))));
  const int groups = kThreads / g;
  const int sub = tid % g;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    ++sweeps;
    if (tid == 0) *flag_sh = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      for (int base = 0; base < np; base += groups) {
        const int pi = base + tid / g;
        int p = 0, q = k;
        if (pi < np) {
          const int a = (pi == 0) ? 0 : ((round + pi - 1) % (ne - 1)) + 1;
          const int b = ((round + ne - 1 - pi - 1) % (ne - 1)) + 1;
          p = a < b ? a : b;
          q = a < b ? b : a;
        }
        const bool active = pi < np && q < k;
        jacobi_pair<R, V, NV>(Z + (size_t)p * ldz, Z + (size_t)(active ? q : p) * ldz, n, sub, g, active, tol, floor2,
                              flag_sh);
      }
      __syncthreads();
    }
    const int f = *flag_sh;
    __syncthreads();
    if (!f) break;
  }
  return sweeps;
}

// The same sweeps without register blocking (rows too long for the registers of a group): two passes
// over shared or global memory per pair.
template <typename R>
__device__ inline int jacobi_sweeps_loop(int k, int n, R* Z, int ldz, int max_sweeps, R tol, R floor2, int* flag_sh) {
  const int tid = threadIdx.x;
  const int ne = k + (k & 1), np = ne / 2;
  int g = kThreads / np;
  g = g >= 32 ? 32 : (g >= 16 ? 16 : (g >= 8 ? 8 : (g >= 4 ? 4 : (g >= 2 ? 2 : 1))));
  const int groups = kThreads / g;
  const int sub = tid % g;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    ++sweeps;
    if (tid == 0) *flag_sh = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      for (int base = 0; base < np; base += groups) {
        const int pi = base + tid / g;
        int p = 0, q = k;
        if (pi < np) {
          const int a = (pi == 0) ? 0 : ((round + pi - 1) % (ne - 1)) + 1;
          const int b = ((round + ne - 1 - pi - 1) % (ne - 1)) + 1;
          p = a < b ? a : b;
          q = a < b ? b : a;
        }
        const bool active = pi < np && q < k;
        R al = R(0), be = R(0), ga = R(0);
        R* zp = Z + (size_t)p * ldz;
        R* zq = Z + (size_t)(active ? q : p) * ldz;
        if (active) {
          for (int e = sub; e < n; e += g) {
            const R x = zp[e], y = zq[e];
            al += x * x;
            be += y * y;
            ga += x * y;
          }
        }
        for (int o = g >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (active && al > floor2 && be > floor2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const R zeta = (be - al) / (R(2) * ga);
          const R az = fabs(zeta);
          const R den = az > R(1) ? az * (R(1) + sqrt(R(1) + (R(1) / az) * (R(1) / az))) : az + sqrt(R(1) + az * az);
          const R t = (zeta >= R(0) ? R(1) : R(-1)) / den;
          const R c = R(1) / sqrt(R(1) + t * t);
          const R s = c * t;
          for (int e = sub; e < n; e += g) {
            const R x = zp[e], y = zq[e];
            zp[e] = c * x - s * y;
            zq[e] = s * x + c * y;
          }
          if (sub == 0) *flag_sh = 1;
        }
      }
      __syncthreads();
    }
    const int f = *flag_sh;
    __syncthreads();
    if (!f) break;
  }
  return sweeps;
}

// The rows are first scaled so that the largest has unit norm (a common scale changes no singular
// direction). floor_rel: a row whose norm is at most floor_rel (relative to the largest) is not
// rotated; its singular value is zero at the working precision, and the caller must drop it (its
// direction is not orthogonalised). floor_rel keeps such rows far from underflow, where their
// inner products lose all relative precision and the sweep would not converge.
template <typename R>
__device__ int cta_onesided_jacobi(int k, int n, R* Z, int ldz, R* nrm2, R* max_nrm2, int max_sweeps, R tol,
                                   R floor_rel, int* flag_sh, R* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int sweeps = 0;
  R loc = R(0);
  for (int j = warp; j < k; j += kWarps) {
    const R* z = Z + (size_t)j * ldz;
    R acc = R(0);
    for (int e = lane; e < n; e += 32) acc += z[e] * z[e];
    acc = warp_sum(acc);
    loc = fmax(loc, acc);
  }
  const R mx0 = block_max(loc, red);
  if (mx0 > R(0)) {
    const R inv = R(1) / sqrt(mx0);
    for (int j = warp; j < k; j += kWarps) {
      R* z = Z + (size_t)j * ldz;
      for (int e = lane; e < n; e += 32) z[e] *= inv;
    }
    __syncthreads();
  }
  const R floor2 = floor_rel * floor_rel;
  if (k > 1) {
    const int np = (k + (k & 1)) / 2;
    int g = kThreads / np;
    g = g >= 32 ? 32 : (g >= 16 ? 16 : (g >= 8 ? 8 : (g >= 4 ? 4 : (g >= 2 ? 2 : 1))));
    bool done = false;
    if constexpr (sizeof(R) == 4) {
      // float rows of a length and leading dimension that are multiples of 4: float4 vectors,
      // up to 8 per thread (n <= 32 g)
      if ((n & 3) == 0 && (ldz & 3) == 0 && n <= 32 * g) {
        sweeps = jacobi_sweeps<R, 4, 8>(k, n, Z, ldz, max_sweeps, tol, floor2, flag_sh);
        done = true;
      }
    }
    if (!done) {
      if (n <= 16 * g) sweeps = jacobi_sweeps<R, 1, 16>(k, n, Z, ldz, max_sweeps, tol, floor2, flag_sh);
      else sweeps = jacobi_sweeps_loop<R>(k, n, Z, ldz, max_sweeps, tol, floor2, flag_sh);
    }
  }
  R mx = R(0);
  for (int j = warp; j < k; j += kWarps) {
    const R* z = Z + (size_t)j * ldz;
    R acc = R(0);
    for (int e = lane; e < n; e += 32) acc += z[e] * z[e];
    acc = warp_sum(acc);
    if (lane == 0) nrm2[j] = acc;
    mx = fmax(mx, acc);
  }
  mx = block_max(mx, red);
  if (tid == 0) *max_nrm2 = mx;
  __syncthreads();
  return sweeps;
}

// rank[i] = position of v[i] in descending order (ties by index).
template <typename R>
__device__ void cta_rank_desc_vec(int n, const R* v, int* rank) {
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const R wi = v[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const R wj = v[j];
      r += (wj > wi) || (wj == wi && j < i);
    }
    rank[i] = r;
  }
  __syncthreads();
}

}  // namespace tnmc
