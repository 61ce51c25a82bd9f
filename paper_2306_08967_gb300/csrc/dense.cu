// Dense building blocks on n x d (tall-skinny) arrays: GEMM with a small right factor,
// Gram matrices, Cholesky with triangular inverse, and the adjacency SpMM.  Used by the
// randomized t-SVD initialisation (Appendix A, Algorithm 3; Halko et al.), the query
// (Sec. 4.6) and the periodic fold of the transforms into the bases.
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "damf_internal.cuh"
#include "tc_gemm.cuh"

namespace damf {

// cuTensorMapEncodeTiled from the driver (the library links only the runtime), or null.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The 4-D view of A (n x K, row-major, lda floats per row) that k_gemm_tc_tma loads from:
// [n / 8 row groups][K / 4 column groups][8 rows][4 floats], strides 8 lda, 16 bytes and lda
// floats, box 16 x 4 x 8 x 4 = one 128-row by 16-column chunk in the MMA's canonical layout.
// False when A does not meet the tensor map's alignment rules or the encoder is missing.
static bool gemm_tensor_map(CUtensorMap* m, const float* A, int lda, long long n, int K) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || n < 8 || (reinterpret_cast<uintptr_t>(A) & 15u) != 0 || (lda & 3) != 0 || K % tc::kTmaChunk != 0)
    return false;
  const cuuint64_t dims[4] = {4, 8, (cuuint64_t)(K / 4), (cuuint64_t)(n / 8)};
  const cuuint64_t strides[3] = {(cuuint64_t)lda * 4, 16, (cuuint64_t)lda * 4 * 8};
  const cuuint32_t box[4] = {4, 8, (cuuint32_t)(tc::kTmaChunk / 4), (cuuint32_t)(tc::kTileM / 8)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(A), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[n x N] = A[n x K] B[K x N]; 64-row tiles, 16 x 16 threads, each a 4 x (N/16) micro-tile.
// Optional per-column scalings: A's column k by ascale[k] (before), C's column j by cscale[j].
template <int K, int N>
__global__ void __launch_bounds__(256) k_gemm_tall(const float* __restrict__ A, int lda, long long n,
                                                   const float* __restrict__ B, float* __restrict__ C, int ldc,
                                                   const float* __restrict__ ascale, const float* __restrict__ cscale) {
  extern __shared__ float smem[];
  float* Bs = smem;             // K x N
  float* As = smem + K * N;     // 64 x (K + 1)
  constexpr int CN = N / 16;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int i = threadIdx.x; i < K * N; i += 256) Bs[i] = B[i];
  for (long long r0 = (long long)blockIdx.x * 64; r0 < n; r0 += (long long)gridDim.x * 64) {
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * K; i += 256) {
      const int rr = i / K, k = i % K;
      float v = 0.f;
      if (r0 + rr < n) {
        v = A[(r0 + rr) * lda + k];
        if (ascale) v *= ascale[k];
      }
      As[rr * (K + 1) + k] = v;
    }
    __syncthreads();
    float acc[4][CN];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < CN; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      float av[4], bv[CN];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[(ty + 16 * a) * (K + 1) + k];
#pragma unroll
      for (int b = 0; b < CN; ++b) bv[b] = Bs[k * N + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < CN; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const long long row = r0 + ty + 16 * a;
      if (row >= n) continue;
#pragma unroll
      for (int b = 0; b < CN; ++b) {
        const int col = tx + 16 * b;
        C[row * ldc + col] = cscale ? acc[a][b] * cscale[col] : acc[a][b];
      }
    }
  }
}

template <int K, int N>
static cudaError_t gemm_tall_kn(const float* A, int lda, long long n, const float* B, float* C, int ldc,
                                const float* as, const float* cs, cudaStream_t s) {
  const size_t sm = (size_t)(K * N + 64 * (K + 1)) * sizeof(float);
  cudaFuncSetAttribute(k_gemm_tall<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  long long tiles = (n + 63) / 64;
  int grid = (int)(tiles < 152 * 8 ? tiles : 152 * 8);
  if (grid < 1) grid = 1;
  k_gemm_tall<K, N><<<grid, 256, sm, s>>>(A, lda, n, B, C, ldc, as, cs);
  return cudaGetLastError();
}

template <int K, int N>
static cudaError_t gemm_tc_kn(const float* A, int lda, long long n, const float* B, float* C, int ldc,
                              const float* as, const float* cs, int* err, cudaStream_t s) {
  if constexpr (tc::tma_stages<K, N>() >= 2) {
    // TMA-fed kernel: B split once per CTA, A chunks copied by the tensor-memory accelerator
    CUtensorMap m;
    if (gemm_tensor_map(&m, A, lda, n, K)) {
      const size_t smt = tc::tma_smem_bytes<K, N>();
      cudaFuncSetAttribute(tc::k_gemm_tc_tma<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const long long tiles = (n + tc::kTileM - 1) / tc::kTileM;
      const int grid = (int)(tiles < sms ? tiles : sms);
      tc::k_gemm_tc_tma<K, N><<<grid, tc::kThreads, smt, s>>>(m, A, lda, n, B, C, ldc, as, cs, err);
      return cudaGetLastError();
    }
  }
  if constexpr (tc::pipe_smem_bytes<K, N>() <= 227 * 1024) {
    // the pipelined kernel: B split once per CTA, two A stages, one CTA per SM
    const size_t smp = tc::pipe_smem_bytes<K, N>();
    cudaFuncSetAttribute(tc::k_gemm_tc_pipe<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (n + tc::kTileM - 1) / tc::kTileM;
    int grid = (int)(tiles < sms ? tiles : sms);
    if (grid < 1) grid = 1;
    tc::k_gemm_tc_pipe<K, N><<<grid, tc::kThreads, smp, s>>>(A, lda, n, B, C, ldc, as, cs, err);
    return cudaGetLastError();
  }
  const size_t sm = tc::smem_bytes<K, N>();
  cudaFuncSetAttribute(tc::k_gemm_tc<K, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (n + tc::kTileM - 1) / tc::kTileM;
  int grid = (int)(tiles < 2LL * sms ? tiles : 2LL * sms);
  if (grid < 1) grid = 1;
  tc::k_gemm_tc<K, N><<<grid, tc::kThreads, sm, s>>>(A, lda, n, B, C, ldc, as, cs, err);
  return cudaGetLastError();
}

// Tensor-core version (kind::tf32, three-term split) of gemm_tall_scaled; `err` receives 1
// if a bounded wait for the tensor core ran out.
cudaError_t gemm_tall_tc(const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                         const float* ascale, const float* cscale, int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
#define DAMF_GTC(KK, NN) \
  if (K == KK && N == NN) return gemm_tc_kn<KK, NN>(A, lda, n, B, C, ldc, ascale, cscale, err, s);
  DAMF_GTC(32, 32) DAMF_GTC(64, 64) DAMF_GTC(96, 96) DAMF_GTC(128, 128) DAMF_GTC(160, 160)
  DAMF_GTC(32, 16) DAMF_GTC(64, 32) DAMF_GTC(96, 64) DAMF_GTC(160, 128)
#undef DAMF_GTC
  return cudaErrorInvalidValue;
}

cudaError_t gemm_tall_scaled(const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                             const float* ascale, const float* cscale, cudaStream_t s) {
#define DAMF_GT(KK, NN) \
  if (K == KK && N == NN) return gemm_tall_kn<KK, NN>(A, lda, n, B, C, ldc, ascale, cscale, s);
  DAMF_GT(16, 16) DAMF_GT(32, 32) DAMF_GT(64, 64) DAMF_GT(96, 96) DAMF_GT(128, 128) DAMF_GT(160, 160)
  DAMF_GT(32, 16) DAMF_GT(64, 32) DAMF_GT(96, 64) DAMF_GT(160, 128)
#undef DAMF_GT
  return cudaErrorInvalidValue;
}

// n x K by K x N product for a context: tensor cores in mixed precision when the shape is
// covered (K a multiple of 32), otherwise the FP32 SIMT kernel.
cudaError_t gemm_ctx(Ctx* c, const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                     const float* ascale, const float* cscale, cudaStream_t s) {
  if (c->cfg.precision == 1 && K % tc::kChunkK == 0) {
    const cudaError_t e = gemm_tall_tc(A, lda, n, B, K, N, C, ldc, ascale, cscale, &c->hdr->status, s);
    if (e != cudaErrorInvalidValue) return e;
    cudaGetLastError();
  }
  return gemm_tall_scaled(A, lda, n, B, K, N, C, ldc, ascale, cscale, s);
}

cudaError_t gemm_tall(const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                      cudaStream_t s) {
  return gemm_tall_scaled(A, lda, n, B, K, N, C, ldc, nullptr, nullptr, s);
}

// Partial Grams: block b accumulates rows [b*rows_per, (b+1)*rows_per) into part[b] (K x K).
template <int K>
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ A, int lda, long long n,
                                                   long long rows_per, float* part) {
  constexpr int CK = K / 16;
  __shared__ float tile[32][K + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[CK][CK];
#pragma unroll
  for (int a = 0; a < CK; ++a)
#pragma unroll
    for (int b = 0; b < CK; ++b) acc[a][b] = 0.f;
  const long long r_begin = blockIdx.x * rows_per;
  const long long r_end = min(n, r_begin + rows_per);
  for (long long r0 = r_begin; r0 < r_end; r0 += 32) {
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * K; i += 256) {
      const int rr = i / K, k = i % K;
      tile[rr][k] = (r0 + rr < r_end) ? A[(r0 + rr) * lda + k] : 0.0f;
    }
    __syncthreads();
    for (int rr = 0; rr < 32; ++rr) {
      float x[CK], y[CK];
#pragma unroll
      for (int a = 0; a < CK; ++a) x[a] = tile[rr][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < CK; ++b) y[b] = tile[rr][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < CK; ++a)
#pragma unroll
        for (int b = 0; b < CK; ++b) acc[a][b] = fmaf(x[a], y[b], acc[a][b]);
    }
  }
  float* out = part + (size_t)blockIdx.x * K * K;
#pragma unroll
  for (int a = 0; a < CK; ++a)
#pragma unroll
    for (int b = 0; b < CK; ++b) out[(ty + 16 * a) * K + tx + 16 * b] = acc[a][b];
}

__global__ void k_gram_reduce(const float* part, int parts, int KK, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= KK) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += (double)part[(size_t)p * KK + i];
  out[i] = (float)s;
}

cudaError_t gram_tall(Ctx* c, const float* A, int lda, long long n, int K, float* out, cudaStream_t s) {
  int parts = c->ws.gram_parts;
  long long rows_per = (n + parts - 1) / parts;
  rows_per = ((rows_per + 31) / 32) * 32;
  if (rows_per < 32) rows_per = 32;
  parts = (int)((n + rows_per - 1) / rows_per);
  if (parts < 1) parts = 1;
  switch (K) {
    case 16: k_gram_part<16><<<parts, 256, 0, s>>>(A, lda, n, rows_per, c->ws.gram_part); break;
    case 32: k_gram_part<32><<<parts, 256, 0, s>>>(A, lda, n, rows_per, c->ws.gram_part); break;
    case 64: k_gram_part<64><<<parts, 256, 0, s>>>(A, lda, n, rows_per, c->ws.gram_part); break;
    case 96: k_gram_part<96><<<parts, 256, 0, s>>>(A, lda, n, rows_per, c->ws.gram_part); break;
    case 128: k_gram_part<128><<<parts, 256, 0, s>>>(A, lda, n, rows_per, c->ws.gram_part); break;
    case 160: k_gram_part<160><<<parts, 256, 0, s>>>(A, lda, n, rows_per, c->ws.gram_part); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gram_reduce<<<(K * K + 255) / 256, 256, 0, s>>>(c->ws.gram_part, parts, K * K, out);
  return cudaGetLastError();
}

// One CTA: G (K x K, symmetric positive definite) = R^T R with R upper; writes R and R^{-1}.
__global__ void __launch_bounds__(1024) k_chol_inv(const float* __restrict__ G, int K, float* Rout, float* Rinv,
                                                   DevHeader* h) {
  extern __shared__ float smem[];
  float* R = smem;          // K x K
  float* X = smem + K * K;  // K x K
  __shared__ float piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < K * K; i += nt) R[i] = G[i];
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    if (tid == 0) {
      const float p = R[j * K + j];
      piv = p > 0.f ? sqrtf(p) : 0.0f;
      if (!(p > 0.f)) set_status(h, DAMF_ERR_NUMERIC);
    }
    __syncthreads();
    const float ip = piv > 0.f ? 1.0f / piv : 0.0f;
    for (int l = j + tid; l < K; l += nt) R[j * K + l] = (l == j) ? piv : R[j * K + l] * ip;
    __syncthreads();
    const int rem = K - j - 1;
    for (int i = tid; i < rem * rem; i += nt) {
      const int a = j + 1 + i / rem, b = j + 1 + i % rem;
      R[a * K + b] -= R[j * K + a] * R[j * K + b];
    }
    __syncthreads();
  }
  for (int i = tid; i < K * K; i += nt) {
    const int a = i / K, b = i % K;
    if (b < a) R[i] = 0.0f;
    X[i] = (a == b) ? 1.0f : 0.0f;
  }
  __syncthreads();
  // back substitution R X = I, column-parallel
  for (int j = K - 1; j >= 0; --j) {
    for (int col = tid; col < K; col += nt) {
      float s = X[j * K + col];
      for (int l = j + 1; l < K; ++l) s = fmaf(-R[j * K + l], X[l * K + col], s);
      const float p = R[j * K + j];
      X[j * K + col] = p > 0.f ? s / p : 0.0f;
    }
    __syncthreads();
  }
  for (int i = tid; i < K * K; i += nt) {
    if (Rout) Rout[i] = R[i];
    Rinv[i] = X[i];
  }
}

cudaError_t chol_inv_upper2(const float* G, int K, float* R, float* Rinv, DevHeader* h, cudaStream_t s) {
  const size_t sm = (size_t)2 * K * K * sizeof(float);
  cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_chol_inv<<<1, 1024, sm, s>>>(G, K, R, Rinv, h);
  return cudaGetLastError();
}

cudaError_t chol_inv_upper(const float* G, int K, float* Rinv, DevHeader* h, cudaStream_t s) {
  return chol_inv_upper2(G, K, nullptr, Rinv, h, s);
}

// Y[u] = sum_{v in row u} X[v] over an adjacency (the randomized t-SVD's products A Omega,
// A^T Q, A Q'). A row of at most kSpmmLong entries is one warp's (float4 columns, the sum in
// entry order). Longer rows (the hubs of a power-law graph hold millions of entries, and one
// warp per row left a launch waiting seconds on its largest row, its FP32 sum drifting over
// millions of terms) are cut into chunks of kSpmmLong entries, one warp each, whose partial
// sums are then added per row in chunk order: the result is deterministic and each row's sum
// is a sum of short sums.
constexpr int kSpmmLong = 1024;

__global__ void k_spmm(Adj a, int n, const float* __restrict__ X, int l, float* Y) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= n) return;
  const int u = (int)wid;
  const int st = a.start[u], ln = a.len[u];
  if (ln > kSpmmLong) return;   // the chunked pass
  const int nq = l / 4;
  for (int c = lane; c < nq; c += 32) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < ln; ++j) {
      const int v = __ldg(a.col + st + j);
      const float4 x = __ldg(reinterpret_cast<const float4*>(X + (size_t)v * l) + c);
      acc.x += x.x, acc.y += x.y, acc.z += x.z, acc.w += x.w;
    }
    reinterpret_cast<float4*>(Y + (size_t)u * l)[c] = acc;
  }
}

// rows longer than kSpmmLong, appended in any order (the plan sorts them)
__global__ void k_spmm_long_rows(const int32_t* __restrict__ len, int n, int* count, int* rows, int cap) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n || len[u] <= kSpmmLong) return;
  const int i = atomicAdd(count, 1);
  if (i < cap) rows[i] = u;
}

// chunk k = (first entry, entry count) of a long row: its partial sum into P[k]
__global__ void k_spmm_chunks(const int32_t* __restrict__ col, const int2* __restrict__ chunks, int nchunks,
                              const float* __restrict__ X, int l, float* P) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nchunks) return;
  const int2 ch = chunks[wid];
  const int nq = l / 4;
  for (int c = lane; c < nq; c += 32) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < ch.y; ++j) {
      const int v = __ldg(col + ch.x + j);
      const float4 x = __ldg(reinterpret_cast<const float4*>(X + (size_t)v * l) + c);
      acc.x += x.x, acc.y += x.y, acc.z += x.z, acc.w += x.w;
    }
    reinterpret_cast<float4*>(P + (size_t)wid * l)[c] = acc;
  }
}

// long row i (rows[i]) = the sum of its chunks first[i] .. first[i + 1] - 1, in order
__global__ void k_spmm_reduce(const int* __restrict__ rows, const int* __restrict__ first, int nlong,
                              const float* __restrict__ P, int l, float* Y) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nlong) return;
  const int u = rows[wid], k0 = first[wid], k1 = first[wid + 1];
  const int nq = l / 4;
  for (int c = lane; c < nq; c += 32) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = k0; k < k1; ++k) {
      const float4 x = reinterpret_cast<const float4*>(P + (size_t)k * l)[c];
      acc.x += x.x, acc.y += x.y, acc.z += x.z, acc.w += x.w;
    }
    reinterpret_cast<float4*>(Y + (size_t)u * l)[c] = acc;
  }
}

__global__ void k_spmm_gather_rows(const int* __restrict__ rows, int nlong, const int32_t* __restrict__ start,
                                   const int32_t* __restrict__ len, int2* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nlong) out[i] = make_int2(start[rows[i]], len[rows[i]]);
}

void spmm_plan_free(SpmmPlan* p) {
  cudaFree(p->rows);
  cudaFree(p->first);
  cudaFree(p->chunks);
  cudaFree(p->P);
  *p = SpmmPlan{};
}

// The chunks of an adjacency's long rows (setup path: synchronises `s`). Rows in increasing
// order, chunks in entry order, so that the sums do not depend on the order the rows were found.
cudaError_t spmm_plan(const Adj& a, int n, int l, SpmmPlan* p, cudaStream_t s) {
  *p = SpmmPlan{};
  if (n <= 0) return cudaSuccess;
  const long long capl = a.m_cap / kSpmmLong + 1;
  const int cap = (int)(capl < n ? capl : n);
  int* d_count = nullptr;
  int* d_rows = nullptr;
  int2* d_sl = nullptr;
  int count = 0;
  std::vector<int> rows;
  std::vector<int2> sl;
  std::vector<int2> chunks;
  std::vector<int> first;
  cudaError_t e = cudaMalloc(&d_count, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_rows, sizeof(int) * (size_t)cap);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_spmm_long_rows<<<(n + 255) / 256, 256, 0, s>>>(a.len, n, d_count, d_rows, cap);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && count > cap) e = cudaErrorInvalidValue;   // more long rows than entries allow
  if (e == cudaSuccess && count > 0) {
    rows.resize(count);
    sl.resize(count);
    e = cudaMemcpyAsync(rows.data(), d_rows, sizeof(int) * (size_t)count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      std::sort(rows.begin(), rows.end());
      e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMalloc(&d_sl, sizeof(int2) * (size_t)count);
    if (e == cudaSuccess) {
      k_spmm_gather_rows<<<(count + 255) / 256, 256, 0, s>>>(d_rows, count, a.start, a.len, d_sl);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.data(), d_sl, sizeof(int2) * (size_t)count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      first.push_back(0);
      for (int i = 0; i < count; ++i) {
        for (int j = 0; j < sl[i].y; j += kSpmmLong)
          chunks.push_back(make_int2(sl[i].x + j, sl[i].y - j < kSpmmLong ? sl[i].y - j : kSpmmLong));
        first.push_back((int)chunks.size());
      }
      p->nlong = count;
      p->nchunks = (int)chunks.size();
      e = cudaMalloc(&p->rows, sizeof(int) * (size_t)count);
      if (e == cudaSuccess) e = cudaMalloc(&p->first, sizeof(int) * first.size());
      if (e == cudaSuccess) e = cudaMalloc(&p->chunks, sizeof(int2) * chunks.size());
      if (e == cudaSuccess) e = cudaMalloc(&p->P, sizeof(float) * chunks.size() * (size_t)l);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->rows, rows.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->chunks, chunks.data(), sizeof(int2) * chunks.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  cudaFree(d_count);
  cudaFree(d_rows);
  cudaFree(d_sl);
  if (e != cudaSuccess) spmm_plan_free(p);
  return e;
}

cudaError_t spmm(const Adj& a, int n, const float* X, int l, float* Y, const SpmmPlan* plan, cudaStream_t s) {
  const long long threads = (long long)n * 32;
  k_spmm<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, n, X, l, Y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !plan || plan->nchunks == 0) return e;
  const long long tc = (long long)plan->nchunks * 32, tr = (long long)plan->nlong * 32;
  k_spmm_chunks<<<(unsigned)((tc + 255) / 256), 256, 0, s>>>(a.col, plan->chunks, plan->nchunks, X, l, plan->P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_spmm_reduce<<<(unsigned)((tr + 255) / 256), 256, 0, s>>>(plan->rows, plan->first, plan->nlong, plan->P, l, Y);
  return cudaGetLastError();
}

// small K x K product C = A B (one CTA)
__global__ void k_small_mm(const float* A, const float* B, float* C, int K) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < K * K; o += gridDim.x * blockDim.x) {
    const int i = o / K, j = o % K;
    float s = 0.f;
    for (int k = 0; k < K; ++k) s = fmaf(A[i * K + k], B[k * K + j], s);
    C[o] = s;
  }
}

cudaError_t small_mm(const float* A, const float* B, float* C, int K, cudaStream_t s) {
  k_small_mm<<<(K * K + 255) / 256, 256, 0, s>>>(A, B, C, K);
  return cudaGetLastError();
}

}  // namespace damf
