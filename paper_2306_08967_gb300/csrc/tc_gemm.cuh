// Tensor-core GEMM for tall-skinny products C[n x N] = (A[n x K] * diag(ascale)) B[K x N]
// * diag(cscale) on the 5th-generation tensor cores (tcgen05, kind::tf32), FP32 in and out.
//
// Accuracy: each FP32 operand x is split as x = hi + lo with hi = tf32(x) (round to
// nearest) and lo = x - hi (exact); the product uses three MMAs A_hi B_hi + A_hi B_lo +
// A_lo B_hi (error-compensated TF32, Ootomo and Yokota 2022), which keeps the relative
// error near FP32's unit roundoff instead of TF32's 2^-11.
//
// Structure: one CTA of 128 threads per 128-row tile (grid-stride).  For each 32-wide K
// chunk the threads write the hi/lo tiles of A (128 x 32) and B^T (N x 32) into shared
// memory in the canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes), one elected thread issues 4 k-steps x 3 MMAs (M = 128, N, K = 8) accumulating
// in tensor memory, commits them to an mbarrier and all threads wait (bounded).  The
// epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. rows 32w..32w+31 of the tile) and writes C.  In-place use (C == A) is allowed:
// a tile's rows of A are all read before its rows of C are written.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace damf {
namespace tc {

constexpr int kTileM = 128;
constexpr int kChunkK = 32;
constexpr int kThreads = 128;
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, canonical K-major layout without swizzle:
// start address, leading-dimension byte offset (next core matrix along K), stride byte
// offset (next 8-row group), the fixed 0b001 in bits 46-48, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor for kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9,
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) of a rows x kChunkK tile in the canonical layout:
// core matrix (row/8, k/4) at (row/8) * SBO + (k/4) * 128, inside it row%8 * 16 + k%4 * 4
constexpr uint32_t kLBO = 128;                       // next core matrix along K
constexpr uint32_t kSBO = (kChunkK / 4) * 128;       // next 8-row group (1024 bytes)
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(row >> 3) * kSBO + (uint32_t)(k >> 2) * kLBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

template <int K, int N>
__global__ void __launch_bounds__(kThreads) k_gemm_tc(const float* __restrict__ A, int lda, long long n,
                                                      const float* __restrict__ B, float* C, int ldc,
                                                      const float* __restrict__ ascale,
                                                      const float* __restrict__ cscale, int* err) {
  // err: a status word; receives DAMF_ERR_TIMEOUT (5) if a bounded wait ran out
  static_assert(K % kChunkK == 0 && N % 16 == 0 && N >= 16 && N <= 256, "shape");
  constexpr int TMEM_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  constexpr uint32_t A_BYTES = kTileM * kChunkK * 4;   // 16 KB
  constexpr uint32_t B_BYTES = N * kChunkK * 4;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* a_hi = smem;
  unsigned char* a_lo = a_hi + A_BYTES;
  unsigned char* b_hi = a_lo + A_BYTES;
  unsigned char* b_lo = b_hi + B_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  constexpr uint32_t idesc = idesc_tf32(kTileM, N);

  for (long long r0 = (long long)blockIdx.x * kTileM; r0 < n && !failed; r0 += (long long)gridDim.x * kTileM) {
    for (int kc = 0; kc < K; kc += kChunkK) {
      // A: thread = row, 32 consecutive k (8 float4)
      {
        const int row = tid;
        const long long gr = r0 + row;
#pragma unroll
        for (int q = 0; q < kChunkK / 4; ++q) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (gr < n) v = *reinterpret_cast<const float4*>(A + gr * lda + kc + 4 * q);
          if (ascale) {
            v.x *= ascale[kc + 4 * q];
            v.y *= ascale[kc + 4 * q + 1];
            v.z *= ascale[kc + 4 * q + 2];
            v.w *= ascale[kc + 4 * q + 3];
          }
          const float4 h = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
          const float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
          const uint32_t off = tile_off(row, 4 * q);
          *reinterpret_cast<float4*>(a_hi + off) = h;
          *reinterpret_cast<float4*>(a_lo + off) = l;
        }
      }
      // B^T: row = output column j, k from the chunk (B is K x N row-major)
      for (int j = tid; j < N; j += kThreads) {
#pragma unroll
        for (int q = 0; q < kChunkK / 4; ++q) {
          const int k = kc + 4 * q;
          const float4 v = make_float4(B[(size_t)k * N + j], B[(size_t)(k + 1) * N + j], B[(size_t)(k + 2) * N + j],
                                       B[(size_t)(k + 3) * N + j]);
          const float4 h = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
          const float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
          const uint32_t off = tile_off(j, 4 * q);
          *reinterpret_cast<float4*>(b_hi + off) = h;
          *reinterpret_cast<float4*>(b_lo + off) = l;
        }
      }
      // make the generic-proxy writes visible to the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int ks = 0; ks < kChunkK / 8; ++ks) {
          // one k-step of 8 tf32 = two core matrices along K
          const uint32_t koff = (uint32_t)ks * 2 * kLBO;
          const uint64_t dah = smem_desc(smem_u32(a_hi) + koff, kLBO, kSBO);
          const uint64_t dal = smem_desc(smem_u32(a_lo) + koff, kLBO, kSBO);
          const uint64_t dbh = smem_desc(smem_u32(b_hi) + koff, kLBO, kSBO);
          const uint64_t dbl = smem_desc(smem_u32(b_lo) + koff, kLBO, kSBO);
          const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
              :: "r"(tmem), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
              :: "r"(tmem), "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
              :: "r"(tmem), "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&mbar)));
      }
      // bounded wait for the MMAs (they also finish reading the shared tiles)
      {
        long long it = 0;
        uint32_t done = 0;
        while (!done) {
          asm volatile(
              "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
              "selp.u32 %0, 1, 0, p;\n\t}"
              : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase));
          if (!done && ++it > kWaitLimit) {
            failed = 1;
            break;
          }
        }
        phase ^= 1u;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
      if (failed) break;
    }
    if (failed) break;
    // epilogue: warp w reads TMEM lanes 32w..32w+31 = tile rows 32w..32w+31
    const long long row = r0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n) {
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
          float4 o = make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                                 __uint_as_float(v[e + 3]));
          if (cscale) {
            o.x *= cscale[c0 + e];
            o.y *= cscale[c0 + e + 1];
            o.z *= cscale[c0 + e + 2];
            o.w *= cscale[c0 + e + 3];
          }
          *reinterpret_cast<float4*>(C + row * ldc + c0 + e) = o;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (failed) {
    // a wait ran out: wait again (bounded) for the MMAs still in flight before freeing TMEM
    long long it = 0;
    uint32_t done = 0;
    while (!done && ++it <= kWaitLimit) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase ^ 1u));
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
  if (tid == 0 && failed && err) atomicCAS(err, 0, 5);   // 5 = DAMF_ERR_TIMEOUT in the status word
}

template <int K, int N>
constexpr size_t smem_bytes() {
  return (size_t)2 * kTileM * kChunkK * 4 + (size_t)2 * N * kChunkK * 4;
}

}  // namespace tc
}  // namespace damf

namespace damf {
namespace tc {

// Pipelined variant of k_gemm_tc for the fold and full-table queries (K, N <= 160, 2 K N 4 B of
// shared memory for B): the right factor B is split into hi/lo tiles once per CTA for all of K,
// and the rows of A go through two shared-memory stages, so that the threads load and split
// chunk c + 1 of a tile while the tensor core runs the MMAs of chunk c (each stage's MMAs are
// committed to their own mbarrier, which is waited on, bounded, before the stage is refilled).
// One CTA per SM, grid-stride over 128-row tiles; the accumulator is read out per tile as in
// k_gemm_tc. In-place use (C == A) is allowed (a tile's rows of A are read before its rows of
// C are written, and no other CTA touches them).
template <int K, int N>
constexpr size_t pipe_smem_bytes() {
  return (size_t)2 * K * N * 4 + (size_t)2 * 2 * kTileM * kChunkK * 4;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t phase) {
  long long it = 0;
  uint32_t done = 0;
  while (!done) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(smem_u32(mbar)), "r"(phase));
    if (!done && ++it > kWaitLimit) return false;
  }
  return true;
}

template <int K, int N>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc_pipe(const float* __restrict__ A, int lda, long long n,
                                                             const float* __restrict__ B, float* C, int ldc,
                                                             const float* __restrict__ ascale,
                                                             const float* __restrict__ cscale, int* err) {
  static_assert(K % kChunkK == 0 && N % 16 == 0 && N >= 16 && N <= 256, "shape");
  constexpr int NC = K / kChunkK;
  constexpr int TMEM_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  constexpr uint32_t A_BYTES = kTileM * kChunkK * 4;
  constexpr uint32_t B_BYTES = N * kChunkK * 4;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* b_hi = smem;                        // NC chunks of N x 32
  unsigned char* b_lo = b_hi + NC * B_BYTES;
  unsigned char* a_st = b_lo + NC * B_BYTES;         // stage s: hi at a_st + 2 s A_BYTES, lo after it
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])));
    failed = 0;
  }
  // B^T for all of K: row = output column j
  for (int j = tid; j < N; j += kThreads) {
    for (int c = 0; c < NC; ++c) {
#pragma unroll
      for (int q = 0; q < kChunkK / 4; ++q) {
        const int k = c * kChunkK + 4 * q;
        const float4 v = make_float4(B[(size_t)k * N + j], B[(size_t)(k + 1) * N + j], B[(size_t)(k + 2) * N + j],
                                     B[(size_t)(k + 3) * N + j]);
        const float4 hh = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
        const float4 ll = make_float4(v.x - hh.x, v.y - hh.y, v.z - hh.z, v.w - hh.w);
        const uint32_t off = (uint32_t)c * B_BYTES + tile_off(j, 4 * q);
        *reinterpret_cast<float4*>(b_hi + off) = hh;
        *reinterpret_cast<float4*>(b_lo + off) = ll;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(kTileM, N);
  // pend: a commit of stage 0 / 1 not waited for yet; thread 0 waits (bounded), the others learn
  // the outcome at the barrier that follows, so every thread takes the same path
  __shared__ int s_ok;
  int pend0 = 0, pend1 = 0;
  uint32_t ph0 = 0, ph1 = 0;
  bool ok = true;
  long long it = 0;
  for (long long r0 = (long long)blockIdx.x * kTileM; r0 < n && ok; r0 += (long long)gridDim.x * kTileM) {
    const long long gr = r0 + tid;
    for (int c = 0; c < NC && ok; ++c, ++it) {
      const int s = (int)(it & 1);
      // the MMAs that last read this stage are done before it is refilled
      if ((s == 0 && pend0) || (s == 1 && pend1)) {
        if (tid == 0) s_ok = mbar_wait_bounded(&mbar[s], s == 0 ? ph0 : ph1) ? 1 : 0;
        __syncthreads();
        ok = s_ok != 0;
        if (ok && s == 0) {
          ph0 ^= 1u;
          pend0 = 0;
        } else if (ok) {
          ph1 ^= 1u;
          pend1 = 0;
        }
        __syncthreads();   // s_ok is read by everyone before it is written again
      }
      if (!ok) break;
      unsigned char* ahi = a_st + (uint32_t)s * 2 * A_BYTES;
      unsigned char* alo = ahi + A_BYTES;
      const int kc = c * kChunkK;
#pragma unroll
      for (int q = 0; q < kChunkK / 4; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gr < n) v = *reinterpret_cast<const float4*>(A + gr * lda + kc + 4 * q);
        if (ascale) {
          v.x *= ascale[kc + 4 * q];
          v.y *= ascale[kc + 4 * q + 1];
          v.z *= ascale[kc + 4 * q + 2];
          v.w *= ascale[kc + 4 * q + 3];
        }
        const float4 hh = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
        const float4 ll = make_float4(v.x - hh.x, v.y - hh.y, v.z - hh.z, v.w - hh.w);
        const uint32_t off = tile_off(tid, 4 * q);
        *reinterpret_cast<float4*>(ahi + off) = hh;
        *reinterpret_cast<float4*>(alo + off) = ll;
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int ks = 0; ks < kChunkK / 8; ++ks) {
          const uint32_t koff = (uint32_t)ks * 2 * kLBO;
          const uint32_t boff = (uint32_t)c * B_BYTES + koff;
          const uint64_t dah = smem_desc(smem_u32(ahi) + koff, kLBO, kSBO);
          const uint64_t dal = smem_desc(smem_u32(alo) + koff, kLBO, kSBO);
          const uint64_t dbh = smem_desc(smem_u32(b_hi) + boff, kLBO, kSBO);
          const uint64_t dbl = smem_desc(smem_u32(b_lo) + boff, kLBO, kSBO);
          const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
              :: "r"(tmem), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
              :: "r"(tmem), "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
              :: "r"(tmem), "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&mbar[s])));
      }
      if (s == 0) pend0 = 1;
      else pend1 = 1;
    }
    // the tile's MMAs are done: both stages' commits waited for, then the accumulator read out
    if (ok) {
      if (tid == 0) {
        int w = 3;   // bit 0: stage 0 done (or not pending), bit 1: stage 1
        if (pend0 && !mbar_wait_bounded(&mbar[0], ph0)) w &= ~1;
        if ((w & 1) && pend1 && !mbar_wait_bounded(&mbar[1], ph1)) w &= ~2;
        if (!(w & 1)) w &= ~2;   // stage 1 not waited for
        s_ok = w;
      }
      __syncthreads();
      const int w = s_ok;
      ok = w == 3;
      if (pend0 && (w & 1)) {
        ph0 ^= 1u;
        pend0 = 0;
      }
      if (pend1 && (w & 2)) {
        ph1 ^= 1u;
        pend1 = 0;
      }
      __syncthreads();
    }
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const long long row = r0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n) {
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
          float4 o = make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                                 __uint_as_float(v[e + 3]));
          if (cscale) {
            o.x *= cscale[c0 + e];
            o.y *= cscale[c0 + e + 1];
            o.z *= cscale[c0 + e + 2];
            o.w *= cscale[c0 + e + 3];
          }
          *reinterpret_cast<float4*>(C + row * ldc + c0 + e) = o;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (!ok && tid == 0) {
    failed = 1;
    // a wait ran out: wait again (bounded) for the commits still pending before freeing TMEM
    if (pend0) mbar_wait_bounded(&mbar[0], ph0);
    if (pend1) mbar_wait_bounded(&mbar[1], ph1);
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
  if (tid == 0 && failed && err) atomicCAS(err, 0, 5);
}

// TMA-fed variant for the fold, the initialisation and full-table queries. The rows of A reach
// shared memory through the tensor-memory accelerator: a 4-D tensor map views A (n x K,
// row-major, lda) as [row group][k group][row in group][4 floats], so that one
// cp.async.bulk.tensor load of a 128-row x 16-column chunk lands directly in the canonical
// K-major layout of the MMA (core matrices of 8 rows x 16 bytes, 128 bytes apart along K,
// 512 bytes apart along M). S chunk buffers rotate (up to eight, as B leaves room); the copies of
// the next chunks are in flight while the threads split chunk i into hi (in place) and lo
// and the tensor core runs the MMAs of the chunks before it. B is split once per CTA as in k_gemm_tc_pipe. Each stage has
// an mbarrier for its copy (expect-tx) and one for the MMAs that read it (tcgen05.commit).
// Rows of the last partial 8-row group (n % 8 of them) lie outside the tensor map (its row
// extent is n / 8 groups, the rest is filled with zeros) and are read with plain loads.
// Every wait is bounded; on a timeout the CTA waits (bounded) for the copies it issued,
// frees its tensor memory and reports DAMF_ERR_TIMEOUT through `err`.
constexpr int kTmaChunk = 16;                                        // K per chunk
constexpr uint32_t kTmaSBO = (kTmaChunk / 4) * 128;                  // 512: next 8-row group
constexpr uint32_t kTmaChunkBytes = kTileM * kTmaChunk * 4;          // 8 KB per operand buffer

template <int K, int N>
__host__ __device__ constexpr int tma_stages() {
  // B hi/lo for all of K, then hi + lo buffers per stage, within 227 KB of shared memory
  const long long avail = 227LL * 1024 - 2LL * K * N * 4 - 1024;
  const long long s = avail / (2LL * kTmaChunkBytes);
  return s >= 8 ? 8 : (int)s;
}
template <int K, int N>
__host__ __device__ constexpr size_t tma_smem_bytes() {
  return (size_t)2 * K * N * 4 + (size_t)tma_stages<K, N>() * 2 * kTmaChunkBytes;
}

__device__ __forceinline__ uint32_t tile_off16(int row, int k) {   // canonical layout, 16-wide chunk
  return (uint32_t)(row >> 3) * kTmaSBO + (uint32_t)(k >> 2) * kLBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

template <int K, int N>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc_tma(const __grid_constant__ CUtensorMap tmap,
                                                             const float* __restrict__ A, int lda, long long n,
                                                             const float* __restrict__ B, float* C, int ldc,
                                                             const float* __restrict__ ascale,
                                                             const float* __restrict__ cscale, int* err) {
  constexpr int S = tma_stages<K, N>();
  static_assert(S >= 2, "shared memory for two stages");
  static_assert(K % kChunkK == 0 && N % 16 == 0 && N >= 16 && N <= 256, "shape");
  constexpr int NC = K / kTmaChunk;            // chunks per tile
  constexpr int NC32 = K / kChunkK;
  constexpr int TMEM_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  constexpr uint32_t B_BYTES = N * kChunkK * 4;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* b_hi = smem;                  // NC32 chunks of N x 32 (as k_gemm_tc_pipe)
  unsigned char* b_lo = b_hi + NC32 * B_BYTES;
  unsigned char* a_st = b_lo + NC32 * B_BYTES; // stage s: hi at a_st + 2 s kTmaChunkBytes, lo after it
  __shared__ __align__(8) uint64_t full[S];    // the stage's copy landed
  __shared__ __align__(8) uint64_t freed[S];   // the MMAs reading the stage are done
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long tiles = (n + kTileM - 1) / kTileM;
  const long long my_tiles = (long long)blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total = my_tiles * NC;       // chunks this CTA loads
  const long long n8 = n & ~7LL;               // rows covered by the tensor map
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&freed[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  // B^T for all of K: row = output column j
  for (int j = tid; j < N; j += kThreads) {
    for (int c = 0; c < NC32; ++c) {
#pragma unroll
      for (int q = 0; q < kChunkK / 4; ++q) {
        const int k = c * kChunkK + 4 * q;
        const float4 v = make_float4(B[(size_t)k * N + j], B[(size_t)(k + 1) * N + j], B[(size_t)(k + 2) * N + j],
                                     B[(size_t)(k + 3) * N + j]);
        const float4 hh = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
        const float4 ll = make_float4(v.x - hh.x, v.y - hh.y, v.z - hh.z, v.w - hh.w);
        const uint32_t off = (uint32_t)c * B_BYTES + tile_off(j, 4 * q);
        *reinterpret_cast<float4*>(b_hi + off) = hh;
        *reinterpret_cast<float4*>(b_lo + off) = ll;
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(kTileM, N);
  // chunk i of this CTA: tile blockIdx.x + (i / NC) gridDim.x, columns (i % NC) kTmaChunk
  auto issue = [&](long long i) {   // thread 0
    const int st = (int)(i % S);
    const long long t = (long long)blockIdx.x + (i / NC) * gridDim.x;
    const int c = (int)(i % NC);
    unsigned char* dst = a_st + (uint32_t)st * 2 * kTmaChunkBytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(&full[st])), "r"(kTmaChunkBytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(0), "r"(c * (kTmaChunk / 4)),
           "r"((int)(t * (kTileM / 8))), "r"(smem_u32(&full[st]))
        : "memory");
  };
  // s_fail: set (never cleared) when a wait ran out; every thread reads it only after a
  // barrier that follows the last possible write, so all leave together
  long long issued = 0;                        // chunks whose copy was issued (thread 0)
  long long committed = 0;                     // chunks whose MMAs were committed (thread 0)
  if (tid == 0)
    for (; issued < total && issued < S; ++issued) issue(issued);
  for (long long i = 0; i < total; ++i) {
    const int st = (int)(i % S);
    const uint32_t use = (uint32_t)((i / S) & 1);
    const long long t = (long long)blockIdx.x + (i / NC) * gridDim.x;
    const int c = (int)(i % NC);
    const long long r0 = t * kTileM;
    // the chunk's copy has landed: every thread waits on the barrier itself (its acquire is
    // what makes the copy's bytes visible to that thread)
    if (!mbar_wait_bounded(&full[st], use)) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    unsigned char* ahi = a_st + (uint32_t)st * 2 * kTmaChunkBytes;
    unsigned char* alo = ahi + kTmaChunkBytes;
    const long long gr = r0 + tid;
    const int kc = c * kTmaChunk;
#pragma unroll
    for (int q = 0; q < kTmaChunk / 4; ++q) {
      const uint32_t off = tile_off16(tid, 4 * q);
      float4 v;
      if (gr >= n8 && gr < n) v = *reinterpret_cast<const float4*>(A + gr * lda + kc + 4 * q);   // last partial group
      else v = *reinterpret_cast<const float4*>(ahi + off);                                     // zero beyond n
      if (ascale) {
        v.x *= ascale[kc + 4 * q];
        v.y *= ascale[kc + 4 * q + 1];
        v.z *= ascale[kc + 4 * q + 2];
        v.w *= ascale[kc + 4 * q + 3];
      }
      const float4 hh = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
      const float4 ll = make_float4(v.x - hh.x, v.y - hh.y, v.z - hh.z, v.w - hh.w);
      *reinterpret_cast<float4*>(ahi + off) = hh;
      *reinterpret_cast<float4*>(alo + off) = ll;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int ks = 0; ks < kTmaChunk / 8; ++ks) {
        const int g = c * (kTmaChunk / 8) + ks;            // global k-step of 8
        const uint32_t koff = (uint32_t)ks * 2 * kLBO;
        const uint32_t boff = (uint32_t)(g / (kChunkK / 8)) * B_BYTES + (uint32_t)(g % (kChunkK / 8)) * 2 * kLBO;
        const uint64_t dah = smem_desc(smem_u32(ahi) + koff, kLBO, kTmaSBO);
        const uint64_t dal = smem_desc(smem_u32(alo) + koff, kLBO, kTmaSBO);
        const uint64_t dbh = smem_desc(smem_u32(b_hi) + boff, kLBO, kSBO);
        const uint64_t dbl = smem_desc(smem_u32(b_lo) + boff, kLBO, kSBO);
        const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem), "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem), "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem), "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&freed[st])));
      committed = i + 1;
      // refill the stage of chunk i - L with chunk i - L + S once the MMAs of chunk i - L are
      // done: committed L iterations ago, they are normally finished, so thread 0 does not
      // wait on the tensor core, and the copies run S - L chunks ahead of their use
      constexpr int L = S >= 3 ? 2 : 1;
      if (i >= L && issued < total) {
        const long long pi = i - L;
        if (mbar_wait_bounded(&freed[pi % S], (uint32_t)((pi / S) & 1))) issue(issued++);
        else s_fail = 1;
      }
    }
    if (c == NC - 1) {
      // the tile's MMAs are done (its last commit), then the accumulator is read out
      if (tid == 0 && !s_fail && !mbar_wait_bounded(&freed[st], use)) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const long long row = r0 + warp * 32 + lane;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (row < n) {
#pragma unroll
          for (int e = 0; e < 16; e += 4) {
            float4 o = make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                                   __uint_as_float(v[e + 3]));
            if (cscale) {
              o.x *= cscale[c0 + e];
              o.y *= cscale[c0 + e + 1];
              o.z *= cscale[c0 + e + 2];
              o.w *= cscale[c0 + e + 3];
            }
            *reinterpret_cast<float4*>(C + row * ldc + c0 + e) = o;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
  }
  const bool failed = s_fail != 0;   // read after the loop's last barrier by every thread
  if (failed && tid == 0) {
    // a wait ran out: wait (bounded) for the newest copy issued on each stage and for the
    // newest commit before the shared and tensor memory are given up
    for (long long i = issued > S ? issued - S : 0; i < issued; ++i)
      mbar_wait_bounded(&full[i % S], (uint32_t)((i / S) & 1));
    if (committed > 0) {
      const long long li = committed - 1;
      mbar_wait_bounded(&freed[li % S], (uint32_t)((li / S) & 1));
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS));
  if (tid == 0 && failed && err) atomicCAS(err, 0, 5);
}

}  // namespace tc
}  // namespace damf
