// CTA-cooperative dense linear algebra on small matrices: tiled GEMM and a
// cyclic Jacobi eigensolver for symmetric matrices. Every routine is called by
// all threads of the CTA and ends with a barrier.
#pragma once

#include "common.cuh"

namespace tnmc {

template <typename R>
struct GemmSmem {
  R a[16][68];
  R b[16][68];
};

// C[M x N] = alpha * op(A) * op(B) + beta * C, row-major with leading dims.
// op(A)[i][k] = ta ? A[k*lda + i] : A[i*lda + k]; op(B)[k][j] = tb ? B[j*ldb + k] : B[k*ldb + j].
// beta == 0 never reads C. Thread (ty, tx) of a 16x16 grid owns rows ty + 16 i and
// columns tx + 16 j of each 64 x 64 output tile.
template <typename R, typename Acc = R>
__device__ void cta_gemm(int M, int N, int K, R alpha, const R* A, int lda, bool ta, const R* B, int ldb,
                         bool tb, R beta, R* C, int ldc, GemmSmem<R>& sm) {
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  for (int m0 = 0; m0 < M; m0 += 64) {
    for (int n0 = 0; n0 < N; n0 += 64) {
      Acc acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);
      for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += kThreads) {
          int kk, mm;
          if (ta) { kk = e >> 6; mm = e & 63; } else { mm = e >> 4; kk = e & 15; }
          const int gm = m0 + mm, gk = k0 + kk;
          R v = R(0);
          if (gm < M && gk < K) v = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
          sm.a[kk][mm] = v;
        }
        for (int e = tid; e < 16 * 64; e += kThreads) {
          int kk, nn;
          if (tb) { nn = e >> 4; kk = e & 15; } else { kk = e >> 6; nn = e & 63; }
          const int gn = n0 + nn, gk = k0 + kk;
          R v = R(0);
          if (gn < N && gk < K) v = tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
          sm.b[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          Acc av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = (Acc)sm.a[kk][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = (Acc)sm.b[kk][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gn = n0 + tx + 16 * j;
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

struct JacobiSmem {
  int p[128];
  int q[128];
  double c[128];
  double s[128];
  int flag;
};

// Cyclic Jacobi for a symmetric n x n matrix A (lda), n <= 256. On return the
// diagonal of A holds the eigenvalues and the columns of V (ldv) the
// eigenvectors. Rotations follow the symmetric 2x2 Schur decomposition of
// Golub & Van Loan (sym.schur2); pairs are scheduled with the round-robin
// (circle) ordering so that each round's rotations act on disjoint index
// pairs and run in parallel. Stops after a sweep without a rotation that is
// significant relative to sqrt(|a_pp a_qq|), or after max_sweeps.
template <typename R>
__device__ void cta_jacobi_eig(int n, R* A, int lda, R* V, int ldv, int max_sweeps, JacobiSmem& js) {
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += kThreads) {
    const int i = e / n, j = e % n;
    V[(size_t)i * ldv + j] = (i == j) ? R(1) : R(0);
  }
  __syncthreads();
  if (n <= 1) return;
  const int ne = n + (n & 1);
  const int np = ne / 2;
  const R tol = R(4) * Eps<R>::v;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) js.flag = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      for (int i = tid; i < np; i += kThreads) {
        // circle method: player 0 fixed, the others rotate by `round`
        const int a = (i == 0) ? 0 : ((round + i - 1) % (ne - 1)) + 1;
        const int b = ((round + ne - 1 - i - 1) % (ne - 1)) + 1;
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < n) {
          const R apq = A[(size_t)p * lda + q];
          const R app = A[(size_t)p * lda + p];
          const R aqq = A[(size_t)q * lda + q];
          const R thr = tol * sqrt(fabs(app * aqq));
          if (apq != R(0) && fabs(apq) > thr * R(1e-3)) {
            if (fabs(apq) > thr) js.flag = 1;
            const R tau = (aqq - app) / (R(2) * apq);
            const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
            const R cc = R(1) / sqrt(R(1) + t * t);
            c = cc;
            s = t * cc;
          }
        } else {
          p = -1;
        }
        js.p[i] = p;
        js.q[i] = q;
        js.c[i] = c;
        js.s[i] = s;
      }
      __syncthreads();
      // A <- A J and V <- V J (columns p, q of each pair)
      for (int e = tid; e < np * n; e += kThreads) {
        const int i = e / n, row = e % n;
        const int p = js.p[i];
        if (p < 0 || js.s[i] == 0.0) continue;
        const int q = js.q[i];
        const R c = (R)js.c[i], s = (R)js.s[i];
        R* ar = A + (size_t)row * lda;
        const R x = ar[p], y = ar[q];
        ar[p] = c * x - s * y;
        ar[q] = s * x + c * y;
        R* vr = V + (size_t)row * ldv;
        const R vx = vr[p], vy = vr[q];
        vr[p] = c * vx - s * vy;
        vr[q] = s * vx + c * vy;
      }
      __syncthreads();
      // A <- J^T A (rows p, q of each pair)
      for (int e = tid; e < np * n; e += kThreads) {
        const int i = e / n, col = e % n;
        const int p = js.p[i];
        if (p < 0 || js.s[i] == 0.0) continue;
        const int q = js.q[i];
        const R c = (R)js.c[i], s = (R)js.s[i];
        const R x = A[(size_t)p * lda + col], y = A[(size_t)q * lda + col];
        A[(size_t)p * lda + col] = c * x - s * y;
        A[(size_t)q * lda + col] = s * x + c * y;
      }
      __syncthreads();
    }
    const int f = js.flag;
    __syncthreads();
    if (!f) break;
  }
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
