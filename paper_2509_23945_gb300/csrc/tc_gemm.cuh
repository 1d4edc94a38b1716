// CTA-cooperative GEMM on the tensor cores for the FP32 path (warp-level mma.sync).
//
// C[M x N] = alpha * op(A) * op(B) + beta * C with the operand conventions of
// cta_gemm (row-major, op = optional transpose, beta == 0 never reads C). The
// 64 x 64 output tile is split over the 8 warps as 2 x 4 warp tiles of 32 x 16
// (2 x 2 mma tiles of 16 x 8); K advances in chunks of 16 staged through shared
// memory.
//   TC_TF32X3: each FP32 operand is split a = a_hi + a_lo with a_hi, a_lo TF32,
//              and a*b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi (the a_lo b_lo term is
//              below FP32 rounding), accumulated in FP32: FP32-level accuracy.
//   TC_BF16:   one BF16 x BF16 -> FP32 product per term (BF16 inputs).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace tnmc {

// Engines of the environment pass's contractions (the values of TNMC_GEMM_*).
enum GemmMode : int { GEMM_FFMA = 0, GEMM_TF32X3 = 1, GEMM_BF16 = 2, GEMM_UMMA_TF32X3 = 3, GEMM_UMMA_BF16 = 4 };

struct TcGemmSmem {
  // TF32 path: [k][m] / [k][n] FP32 staging (72 = 64 + 8 pad: conflict-free fragment loads)
  // BF16 path: [m][k] / [n][k] BF16 pairs (24 = 16 + 8 pad)
  union {
    struct { float a[16][72]; float b[16][72]; } f;
    struct { __nv_bfloat16 a[64][24]; __nv_bfloat16 b[64][24]; } h;
  };
};

__device__ inline uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ inline void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ inline void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ inline void cta_gemm_tc(int mode, int M, int N, int K, float alpha, const float* A, int lda, bool ta,
                            const float* B, int ldb, bool tb, float beta, float* C, int ldc, TcGemmSmem& sm) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int wm = (warp >> 2) * 32, wn = (warp & 3) * 16;   // warp tile origin inside the 64 x 64 tile
  for (int m0 = 0; m0 < M; m0 += 64) {
    for (int n0 = 0; n0 < N; n0 += 64) {
      float acc[2][2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int t = 0; t < 4; ++t) acc[i][j][t] = 0.0f;
      for (int k0 = 0; k0 < K; k0 += 16) {
        // stage the 64 x 16 slice of op(A) and the 16 x 64 slice of op(B)
        for (int e = tid; e < 16 * 64; e += kThreads) {
          int kk, mm;
          if (ta) { kk = e >> 6; mm = e & 63; } else { mm = e >> 4; kk = e & 15; }
          const int gm = m0 + mm, gk = k0 + kk;
          float v = 0.0f;
          if (gm < M && gk < K) v = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
          if (mode == GEMM_BF16) sm.h.a[mm][kk] = __float2bfloat16_rn(v);
          else sm.f.a[kk][mm] = v;
        }
        for (int e = tid; e < 16 * 64; e += kThreads) {
          int kk, nn;
          if (tb) { nn = e >> 4; kk = e & 15; } else { kk = e >> 6; nn = e & 63; }
          const int gn = n0 + nn, gk = k0 + kk;
          float v = 0.0f;
          if (gn < N && gk < K) v = tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
          if (mode == GEMM_BF16) sm.h.b[nn][kk] = __float2bfloat16_rn(v);
          else sm.f.b[kk][nn] = v;
        }
        __syncthreads();
        if (mode == GEMM_BF16) {
          uint32_t af[2][4], bf[2][2];
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int r0 = wm + i * 16 + gid;
            af[i][0] = *reinterpret_cast<const uint32_t*>(&sm.h.a[r0][tig * 2]);
            af[i][1] = *reinterpret_cast<const uint32_t*>(&sm.h.a[r0 + 8][tig * 2]);
            af[i][2] = *reinterpret_cast<const uint32_t*>(&sm.h.a[r0][tig * 2 + 8]);
            af[i][3] = *reinterpret_cast<const uint32_t*>(&sm.h.a[r0 + 8][tig * 2 + 8]);
          }
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int c0 = wn + j * 8 + gid;
            bf[j][0] = *reinterpret_cast<const uint32_t*>(&sm.h.b[c0][tig * 2]);
            bf[j][1] = *reinterpret_cast<const uint32_t*>(&sm.h.b[c0][tig * 2 + 8]);
          }
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        } else {
#pragma unroll
          for (int ks = 0; ks < 16; ks += 8) {
            uint32_t ah[2][4], al[2][4], bh[2][2], bl[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
              const int r0 = wm + i * 16 + gid;
              const float x[4] = {sm.f.a[ks + tig][r0], sm.f.a[ks + tig][r0 + 8], sm.f.a[ks + tig + 4][r0],
                                  sm.f.a[ks + tig + 4][r0 + 8]};
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                ah[i][t] = to_tf32(x[t]);
                al[i][t] = to_tf32(x[t] - __uint_as_float(ah[i][t]));
              }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int c0 = wn + j * 8 + gid;
              const float y[2] = {sm.f.b[ks + tig][c0], sm.f.b[ks + tig + 4][c0]};
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                bh[j][t] = to_tf32(y[t]);
                bl[j][t] = to_tf32(y[t] - __uint_as_float(bh[j][t]));
              }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                mma_tf32(acc[i][j], al[i], bh[j]);
                mma_tf32(acc[i][j], ah[i], bl[j]);
                mma_tf32(acc[i][j], ah[i], bh[j]);
              }
          }
        }
        __syncthreads();
      }
      // write back: accumulator t of mma tile (i, j) sits at row gid (+8 for t >= 2), column 2 tig (+1)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int gm = m0 + wm + i * 16 + gid + (t >= 2 ? 8 : 0);
            const int gn = n0 + wn + j * 8 + tig * 2 + (t & 1);
            if (gm < M && gn < N) {
              float* c = C + (size_t)gm * ldc + gn;
              const float v = alpha * acc[i][j][t];
              *c = (beta == 0.0f) ? v : v + beta * (*c);
            }
          }
    }
  }
  __syncthreads();
}

}  // namespace tnmc
