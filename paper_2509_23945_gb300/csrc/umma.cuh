// CTA-cooperative GEMM on the Blackwell tensor cores (tcgen05.mma, accumulator in tensor memory).
//
// C[M x N] = alpha * op(A) * op(B) + beta * C, with the operand conventions of cta_gemm
// (row-major, op = optional transpose, beta == 0 never reads C). All 256 threads of the CTA call it.
//
// Output tiles are 128 x 64: one tcgen05.mma of shape M = 128, N = 64 per K step writes the FP32
// accumulator into 64 columns of tensor memory (TMEM lane i = tile row i). K advances in chunks of
// 64 bytes per row (16 TF32 or 32 BF16 values): every thread converts its share of op(A) and op(B)
// from global memory into shared memory, in the no-swizzle K-major layout the MMA reads (8 x 16-byte
// core matrices, 128 bytes each; consecutive K core matrices 128 bytes apart, consecutive 8-row
// groups 512 bytes apart). One elected thread issues the MMAs and commits them to an mbarrier; the
// loads of the next chunk are in flight meanwhile. The epilogue reads the accumulator with
// tcgen05.ld (warp w: lanes 32 (w mod 4) .. + 31, columns 32 (w / 4) .. + 31).
//   UMMA_TF32X3: a = a_hi + a_lo with a_hi, a_lo exact TF32 values (round to nearest), and
//                a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi (a_lo b_lo is below FP32 rounding): three
//                kind::tf32 MMAs into one FP32 accumulator, FP32-level accuracy.
//   UMMA_BF16:   BF16 operands (round to nearest), one kind::f16 MMA per K step, FP32 accumulator.
// Tensor memory is allocated (64 columns) at the start of each call and freed at its end, so no
// TMEM outlives a call. Every wait on the mbarrier is bounded: when one expires the call latches
// ST_TIMEOUT into *status, skips the rest of its work and still frees its TMEM.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace tnmc {

constexpr int kUmmaM = 128;                 // tile rows (TMEM lanes)
constexpr int kUmmaN = 64;                  // tile columns (TMEM columns, 32-bit each)
constexpr int kUmmaRowBytes = 64;           // bytes of one staged row per K chunk
constexpr int kUmmaCoreBytes = 128;         // one core matrix: 8 rows x 16 bytes
constexpr int kUmmaLbo = kUmmaCoreBytes;    // next core matrix along K
constexpr int kUmmaSbo = 8 * kUmmaRowBytes; // next 8-row group
constexpr int kUmmaABytes = kUmmaM * kUmmaRowBytes;   // 8 KB
constexpr int kUmmaBBytes = kUmmaN * kUmmaRowBytes;   // 4 KB
// Shared-memory staging per call: TF32x3 holds hi and lo copies of both operands.
constexpr int kUmmaStageBytes = 2 * (kUmmaABytes + kUmmaBBytes);   // 24 KB
constexpr long long kUmmaWaitCycles = 4000000000LL;                 // about 2 s at 2 GHz

enum UmmaKind : int { UMMA_TF32X3 = 0, UMMA_BF16 = 1 };

// Control words of one call: the mbarrier the MMAs commit to, the TMEM base address written by
// tcgen05.alloc, and the abort flag set when a wait expired.
struct __align__(8) UmmaCtl {
  unsigned long long mbar;
  uint32_t taddr;
  int abort;
};

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row group) byte
// offsets, all in 16-byte units; descriptor version 1 (bits 46-47); no swizzle (bits 61-63 = 0).
__device__ inline uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32 / kind::f16: D in FP32 (bits 4-5 = 1), A and B formats
// (bits 7-9, 10-12: TF32 = 2, BF16 = 1), both K-major (bits 15, 16 = 0), N / 8 (bits 17-22),
// M / 16 (bits 24-28).
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kUmmaN >> 3) << 17) | ((uint32_t)(kUmmaM >> 4) << 24);
}

__device__ inline void umma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem), "l"(ad), "l"(bd), "r"(umma_idesc(2)), "r"(acc)
      : "memory");
}

__device__ inline void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem), "l"(ad), "l"(bd), "r"(umma_idesc(1)), "r"(acc)
      : "memory");
}

__device__ inline void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory stores made visible to the tensor cores (async proxy).
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait for the given phase parity of an mbarrier; false when the wait expired.
__device__ inline bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kUmmaWaitCycles) return false;
  }
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ inline void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Byte offset of element (row i, byte b of the row's K chunk) in the no-swizzle K-major layout.
__device__ inline int umma_off(int i, int b) {
  return (i >> 3) * kUmmaSbo + (b >> 4) * kUmmaCoreBytes + (i & 7) * 16 + (b & 15);
}

__device__ inline float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// stage: kUmmaStageBytes of shared memory, 128-byte aligned. ctl: control words in shared memory.
// status: device status word (ST_TIMEOUT on an expired wait). M, N, K >= 0.
// Not inlined: its registers stay out of the callers' allocation (the slice kernel runs at 128).
template <int KIND>
__device__ __noinline__ void cta_gemm_umma(int M, int N, int K, float alpha, const float* A, int lda, bool ta, const float* B,
                              int ldb, bool tb, float beta, float* C, int ldc, unsigned char* stage, UmmaCtl& ctl,
                              unsigned int* status) {
  constexpr bool X3 = KIND == UMMA_TF32X3;
  constexpr int ESZ = X3 ? 4 : 2;                     // bytes per staged element
  constexpr int KC = kUmmaRowBytes / ESZ;             // K elements per chunk: 16 (TF32) or 32 (BF16)
  constexpr int KSTEP = 32;                           // bytes of K per MMA (K = 8 TF32 or 16 BF16)
  constexpr int PA = kUmmaM * KC / kThreads;          // op(A) elements each thread stages per chunk
  constexpr int PB = kUmmaN * KC / kThreads;          // op(B) elements
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* sA = stage;
  unsigned char* sB = stage + kUmmaABytes;
  unsigned char* sA2 = stage + kUmmaABytes + kUmmaBBytes;   // lo parts (TF32x3)
  unsigned char* sB2 = sA2 + kUmmaABytes;
  const uint32_t mbar = smem_u32(&ctl.mbar);

  if (warp == 0)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl.taddr)),
                 "r"(kUmmaN)
                 : "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ctl.abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl.taddr;
  uint32_t phase = 0;
  bool ok = true;

  float ra[PA], rb[PB];
  auto fetch = [&](int m0, int n0, int k0) {
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int e = tid + t * kThreads;
      int i, k;
      if (ta) { k = e / kUmmaM; i = e % kUmmaM; } else { i = e / KC; k = e % KC; }
      const int gm = m0 + i, gk = k0 + k;
      ra[t] = (gm < M && gk < K) ? (ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < PB; ++t) {
      const int e = tid + t * kThreads;
      int j, k;
      if (tb) { j = e / KC; k = e % KC; } else { k = e / kUmmaN; j = e % kUmmaN; }
      const int gn = n0 + j, gk = k0 + k;
      rb[t] = (gn < N && gk < K) ? (tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]) : 0.0f;
    }
  };
  auto put = [&](unsigned char* hi, unsigned char* lo, int off, float v) {
    if constexpr (X3) {
      const float h = tf32_rn(v);
      *reinterpret_cast<float*>(hi + off) = h;
      *reinterpret_cast<float*>(lo + off) = tf32_rn(v - h);
    } else {
      *reinterpret_cast<__nv_bfloat16*>(hi + off) = __float2bfloat16_rn(v);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int e = tid + t * kThreads;
      int i, k;
      if (ta) { k = e / kUmmaM; i = e % kUmmaM; } else { i = e / KC; k = e % KC; }
      put(sA, sA2, umma_off(i, k * ESZ), ra[t]);
    }
#pragma unroll
    for (int t = 0; t < PB; ++t) {
      const int e = tid + t * kThreads;
      int j, k;
      if (tb) { j = e / KC; k = e % KC; } else { k = e / kUmmaN; j = e % kUmmaN; }
      put(sB, sB2, umma_off(j, k * ESZ), rb[t]);
    }
  };
  auto wait = [&]() {
    if (!mbar_wait_bounded(mbar, phase)) {
      ctl.abort = 1;
      atomicOr(status, (unsigned int)ST_TIMEOUT);
    }
    phase ^= 1u;
  };

  const int nk = (K + KC - 1) / KC;
  for (int m0 = 0; m0 < M && ok; m0 += kUmmaM) {
    for (int n0 = 0; n0 < N && ok; n0 += kUmmaN) {
      if (nk > 0) fetch(m0, n0, 0);
      for (int c = 0; c < nk; ++c) {
        if (c > 0) wait();   // the MMAs of chunk c - 1 have read the staging buffers
        stash();
        fence_async_smem();
        __syncthreads();
        if (ctl.abort) { ok = false; break; }
        if (tid == 0) {
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB), a1 = smem_u32(sA2), b1 = smem_u32(sB2);
#pragma unroll
          for (int s = 0; s < kUmmaRowBytes / KSTEP; ++s) {
            const uint32_t o = s * 2 * kUmmaCoreBytes;
            const uint32_t first = (c > 0 || s > 0) ? 1u : 0u;
            const uint64_t ah = umma_sdesc(a0 + o, kUmmaLbo, kUmmaSbo), bh = umma_sdesc(b0 + o, kUmmaLbo, kUmmaSbo);
            if constexpr (X3) {
              const uint64_t al = umma_sdesc(a1 + o, kUmmaLbo, kUmmaSbo), bl = umma_sdesc(b1 + o, kUmmaLbo, kUmmaSbo);
              umma_tf32(tmem, al, bh, first);
              umma_tf32(tmem, ah, bl, 1u);
              umma_tf32(tmem, ah, bh, 1u);
            } else {
              umma_bf16(tmem, ah, bh, first);
            }
          }
          umma_commit(mbar);
        }
        if (c + 1 < nk) fetch(m0, n0, (c + 1) * KC);   // in flight while the MMAs run
      }
      if (!ok) break;
      if (nk > 0) wait();
      __syncthreads();
      if (ctl.abort) { ok = false; break; }
      tc_fence_after();
      float v[32];
      if (nk > 0) {
        const uint32_t ta0 = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32u * (uint32_t)(warp >> 2);
        tmem_ld16(ta0, v);
        tmem_ld16(ta0 + 16, v + 16);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.0f;
      }
      const int gm = m0 + 32 * (warp & 3) + lane;
      const int gn0 = n0 + 32 * (warp >> 2);
      if (gm < M) {
        float* crow = C + (size_t)gm * ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int gn = gn0 + j;
          if (gn < N) crow[gn] = (beta == 0.0f) ? alpha * v[j] : alpha * v[j] + beta * crow[gn];
        }
      }
      tc_fence_before();
      __syncthreads();   // every TMEM read is done before the next tile's MMAs overwrite the accumulator
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUmmaN) : "memory");
  if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
  __syncthreads();
}

}  // namespace tnmc
