// CTA-cooperative dense linear algebra on small matrices: tiled GEMM and a
// cyclic Jacobi eigensolver for symmetric matrices. Every routine is called by
// all threads of the CTA and ends with a barrier.
#pragma once

#include "common.cuh"

namespace tnmc {

// K-chunk of the CUDA-core GEMM (16: the prefetch registers fit without spills).
template <typename R> struct GemmKC { static constexpr int v = 16; };

template <typename R>
struct __align__(16) GemmSmem {
  R a[GemmKC<R>::v][68];
  R b[GemmKC<R>::v][68];
};

// C[M x N] = alpha * op(A) * op(B) + beta * C, row-major with leading dims.
// op(A)[i][k] = ta ? A[k*lda + i] : A[i*lda + k]; op(B)[k][j] = tb ? B[j*ldb + k] : B[k*ldb + j].
// beta == 0 never reads C. Thread (ty, tx) of a 16x16 grid owns rows 4 ty + i and
// columns 4 tx + j of each 64 x 64 output tile, so each k step reads its four A and four B
// values with one 16-byte shared-memory load each. The next K-chunk is loaded into
// registers while the current one is multiplied out of shared memory, so global
// (L2 / HBM) latency overlaps the arithmetic.
// Four consecutive shared-memory values (16-byte aligned) into registers.
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

template <typename R, typename Acc = R>
__device__ void cta_gemm(int M, int N, int K, R alpha, const R* A, int lda, bool ta, const R* B, int ldb,
                         bool tb, R beta, R* C, int ldc, GemmSmem<R>& sm) {
  constexpr int KC = GemmKC<R>::v;
  constexpr int PER = KC * 64 / kThreads;   // elements of each operand a thread stages per chunk
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  R ra[PER], rb[PER];
  auto fetch = [&](int m0, int n0, int k0) {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = tid + t * kThreads;
      int kk, mm;
      if (ta) { kk = e >> 6; mm = e & 63; } else { mm = e / KC; kk = e % KC; }
      const int gm = m0 + mm, gk = k0 + kk;
      ra[t] = (gm < M && gk < K) ? (ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : R(0);
      int kb, nb;
      if (tb) { nb = e / KC; kb = e % KC; } else { kb = e >> 6; nb = e & 63; }
      const int gn = n0 + nb, gkb = k0 + kb;
      rb[t] = (gn < N && gkb < K) ? (tb ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn]) : R(0);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int e = tid + t * kThreads;
      int kk, mm;
      if (ta) { kk = e >> 6; mm = e & 63; } else { mm = e / KC; kk = e % KC; }
      sm.a[kk][mm] = ra[t];
      int kb, nb;
      if (tb) { nb = e / KC; kb = e % KC; } else { kb = e >> 6; nb = e & 63; }
      sm.b[kb][nb] = rb[t];
    }
  };
  for (int m0 = 0; m0 < M; m0 += 64) {
    for (int n0 = 0; n0 < N; n0 += 64) {
      Acc acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);
      if (K > 0) fetch(m0, n0, 0);
      for (int k0 = 0; k0 < K; k0 += KC) {
        stash();
        __syncthreads();
        if (k0 + KC < K) fetch(m0, n0, k0 + KC);   // in flight while this chunk is multiplied
        const int kend = (K - k0) < KC ? (K - k0) : KC;
        for (int kk = 0; kk < kend; ++kk) {
          Acc av[4], bv[4];
          load4(&sm.a[kk][4 * ty], av);
          load4(&sm.b[kk][4 * tx], bv);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int gm = m0 + 4 * ty + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gn = n0 + 4 * tx + j;
          if (gn >= N) continue;
          R* c = C + (size_t)gm * ldc + gn;
          const R v = alpha * (R)acc[i][j];
          *c = (beta == R(0)) ? v : v + beta * (*c);
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

}  // namespace tnmc
