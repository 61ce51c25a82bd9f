// Link-prediction scores (Sec. 5, "Link Prediction"; appendix "Additional Details of Link
// Prediction"): the score of the node pair (u, v) is the inner product of u's context vector
// with v's content vector, Z[u] . Y[v] with the PPR-enhanced context Z (or X[u] . Y[v] with the
// plain context X); on an undirected graph the larger of the two directions is taken.
//
// In the base representation U = Ub PU, V = Vb PV, X = U Sigma^{1/2}, Y = V Sigma^{1/2} and
// Z = (Zb diag(1/s0)) PU Sigma^{1/2}, so
//     score(u, v) = left(u) G Vb[v]^T,   G = PU diag(sigma) PV^T (d x d),
// with left(u) = Zb[u] diag(1/s0) for the context Z and Ub[u] for X. One d x d matrix G is
// built per call; the bases are read as they are (no n x d query buffers).
//
//   k_score_prep   G (and 1/s0) from PU, PV, sigma, s0                              one CTA
//   k_score_pairs  one row group per pair: q = left(u) G, score = q . Vb[v]         HBM-bound
//   k_topk_scan    per-query top-k over every node v != u: for a slab of candidate rows the
//                  CTA forms the slab x queries score tile, then each warp merges the tile's
//                  scores into its queries' sorted lists; Vb (and left) are read once per
//                  pass of kTopQ queries
//   k_topk_merge   one CTA per query sorts the per-CTA lists (bitonic, 64-bit keys) and
//                  writes the first k
// Keys order by score, then by lower node id: key = (orderable(score) << 32) | ~id.
#include "damf_internal.cuh"

namespace damf {

constexpr int kTopSlab = 64;       // candidate rows per scan step
constexpr int kTopThreads = 512;   // 16 warps: the tiles' shared memory allows one CTA per SM
constexpr int kTopQPT = kTopSlab * kTopQ / kTopThreads;   // queries per thread in the score tile
static_assert(kTopQPT == 4, "the score tile reads one float4 of queries per k");
constexpr int kMergeThreads = 1024;
constexpr int kMergeKeys = 16384;  // per query: scan CTAs x k keys at most

__device__ __forceinline__ unsigned long long topk_key(float s, int id) {
  unsigned u = __float_as_uint(s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned long long)(0xffffffffu - (unsigned)id);
}

__device__ __forceinline__ float key_score(unsigned long long k) {
  const unsigned u = (unsigned)(k >> 32);
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ int key_id(unsigned long long k) { return (int)(0xffffffffu - (unsigned)k); }

// G = PU diag(max(sigma, 0)) PV^T; is0 = 1/s0 (0 where s0 = 0)
__global__ void k_score_prep(const float* PU, const float* PV, const float* sigma, const float* s0, float* G,
                             float* is0, int d) {
  for (int o = threadIdx.x; o < d * d; o += blockDim.x) {
    const int i = o / d, j = o % d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(PU[i * d + k] * fmaxf(sigma[k], 0.f), PV[j * d + k], s);
    G[o] = s;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) is0[k] = s0[k] > 0.f ? 1.0f / s0[k] : 0.0f;
}

// row group (LPR lanes, a float4 each) computes q = a G for its own row a (kept as float4s);
// G is in shared memory, row-major
template <int D>
__device__ __forceinline__ float4 row_times_g(float4 a, const float* Gs, int q, int sub) {
  constexpr int LPR = D / 4;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int i4 = 0; i4 < LPR; ++i4) {
    const int src = sub * LPR + i4;
    const float a0 = __shfl_sync(0xffffffffu, a.x, src), a1 = __shfl_sync(0xffffffffu, a.y, src);
    const float a2 = __shfl_sync(0xffffffffu, a.z, src), a3 = __shfl_sync(0xffffffffu, a.w, src);
    const float av[4] = {a0, a1, a2, a3};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 g = reinterpret_cast<const float4*>(Gs + (size_t)(4 * i4 + c) * D)[q];
      acc.x = fmaf(av[c], g.x, acc.x);
      acc.y = fmaf(av[c], g.y, acc.y);
      acc.z = fmaf(av[c], g.z, acc.z);
      acc.w = fmaf(av[c], g.w, acc.w);
    }
  }
  return acc;
}

template <int LPR>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = 1; o < LPR; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float4 ld4(const float* p, int q) { return __ldg(reinterpret_cast<const float4*>(p) + q); }

__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// scores[p] = left(src[p]) G Vb[dst[p]]^T (symmetric: the max with the (dst, src) direction).
// left = base (Ub or Zb) scaled by `pre` when non-null. Out-of-range ids give 0 and DAMF_ERR_INVALID.
template <int D>
__global__ void __launch_bounds__(256) k_score_pairs(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                     int count, int n, DevHeader* h, const float* __restrict__ G,
                                                     const float* __restrict__ base, const float* __restrict__ pre,
                                                     const float* __restrict__ Vb, int symmetric, float* scores) {
  constexpr int LPR = D / 4, RPW = 32 / LPR;
  extern __shared__ __align__(16) float Gs[];   // [D][D]
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) Gs[i] = G[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, sub = lane / LPR, q = lane % LPR;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const float4 one4 = make_float4(1.f, 1.f, 1.f, 1.f);
  const float4 scale = pre ? ld4(pre, q) : one4;
  for (long long b = gwarp * RPW; b < count; b += nwarps * RPW) {   // warp-uniform
    const long long p = b + sub;
    int u = 0, v = 0;
    bool ok = false;
    if (p < count) {
      u = src[p];
      v = dst[p];
      ok = u >= 0 && u < n && v >= 0 && v < n;
      if (!ok && q == 0) set_status(h, DAMF_ERR_INVALID);
    }
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), yv = a, a2 = a, yu = a;
    if (ok) {
      a = mul4(ld4(base + (size_t)u * D, q), scale);
      yv = ld4(Vb + (size_t)v * D, q);
      if (symmetric) {
        a2 = mul4(ld4(base + (size_t)v * D, q), scale);
        yu = ld4(Vb + (size_t)u * D, q);
      }
    }
    float s = group_sum<LPR>(dot4(row_times_g<D>(a, Gs, q, sub), yv));
    if (symmetric) s = fmaxf(s, group_sum<LPR>(dot4(row_times_g<D>(a2, Gs, q, sub), yu)));
    if (p < count && q == 0) scores[p] = ok ? s : 0.f;
  }
}

// Per query j of this pass: Lq[j] = left(u_j) G (so s1(v) = Vb[v] . Lq[j] = score(u_j, v)) and
// Rq[j] = Vb[u_j] G^T (so s2(v) = left(v) . Rq[j] = score(v, u_j)). One CTA per query.
template <int D>
__global__ void k_topk_queries(const int32_t* __restrict__ rows, int nq, int n, DevHeader* h,
                               const float* __restrict__ G, const float* __restrict__ base,
                               const float* __restrict__ pre, const float* __restrict__ Vb, float* Lq, float* Rq,
                               int32_t* qid) {
  const int j = blockIdx.x;
  int u = rows[j];
  if (u < 0 || u >= n) {
    if (threadIdx.x == 0) set_status(h, DAMF_ERR_INVALID);
    u = -1;
  }
  if (threadIdx.x == 0) qid[j] = u;
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    float l = 0.f, r = 0.f;
    if (u >= 0) {
      for (int k = 0; k < D; ++k) {
        const float b = base[(size_t)u * D + k] * (pre ? pre[k] : 1.f);
        l = fmaf(b, G[k * D + c], l);
        r = fmaf(Vb[(size_t)u * D + k], G[c * D + k], r);
      }
    }
    Lq[j * D + c] = l;
    Rq[j * D + c] = r;
  }
}

// Scan: CTA b takes slabs b, b + grid, ... of kTopSlab candidate rows. Shared memory:
// lists [kTopQ][K] keys sorted in decreasing order; Vs and Ls [kTopSlab][D + 4] the slab's
// rows of Vb and left (row-major, padded so that the 8 rows a warp reads sit in distinct
// banks); Lqt and Rqt [D][kTopQ] the queries' vectors (transposed); S [kTopSlab][kTopQ + 1].
template <int D>
__global__ void __launch_bounds__(kTopThreads) k_topk_scan(int nq, int n, int K, const int32_t* __restrict__ qid,
                                                           const float* __restrict__ Lq, const float* __restrict__ Rq,
                                                           const float* __restrict__ base,
                                                           const float* __restrict__ pre,
                                                           const float* __restrict__ Vb, int symmetric,
                                                           unsigned long long* part) {
  constexpr int LD = D + 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* lists = reinterpret_cast<unsigned long long*>(smem_raw);   // [kTopQ][K]
  float* Vs = reinterpret_cast<float*>(lists + kTopQ * K);                        // [kTopSlab][LD]
  float* Ls = Vs + kTopSlab * LD;                                                 // [kTopSlab][LD]
  float* Lqt = Ls + (symmetric ? kTopSlab * LD : 0);                              // [D][kTopQ]
  float* Rqt = Lqt + D * kTopQ;                                                   // [D][kTopQ]
  float* S = Rqt + (symmetric ? D * kTopQ : 0);                                   // [kTopSlab][kTopQ + 1]
  __shared__ int qs[kTopQ];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kTopQ * K; i += kTopThreads) lists[i] = 0ull;
  for (int i = tid; i < D * kTopQ; i += kTopThreads) {
    const int k = i / kTopQ, j = i % kTopQ;
    Lqt[i] = j < nq ? Lq[j * D + k] : 0.f;
    if (symmetric) Rqt[i] = j < nq ? Rq[j * D + k] : 0.f;
  }
  if (tid < kTopQ) qs[tid] = tid < nq ? qid[tid] : -1;
  const float4 one4 = make_float4(1.f, 1.f, 1.f, 1.f);
  // score tile: thread -> one slab row ti, 4 queries jb .. jb + 3
  const int ti = tid >> 3, jb = (tid & 7) * kTopQPT;
  const long long nslab = ((long long)n + kTopSlab - 1) / kTopSlab;
  for (long long sl = blockIdx.x; sl < nslab; sl += gridDim.x) {
    const long long v0 = sl * kTopSlab;
    __syncthreads();   // the previous tile is merged
    for (int o = tid; o < kTopSlab * (D / 4); o += kTopThreads) {
      const int i = o / (D / 4), c4 = o % (D / 4);
      const long long v = v0 + i;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
      if (v < n) {
        x = ld4(Vb + (size_t)v * D, c4);
        if (symmetric) y = mul4(ld4(base + (size_t)v * D, c4), pre ? ld4(pre, c4) : one4);
      }
      reinterpret_cast<float4*>(Vs + i * LD)[c4] = x;
      if (symmetric) reinterpret_cast<float4*>(Ls + i * LD)[c4] = y;
    }
    __syncthreads();
    float s1[kTopQPT], s2[kTopQPT];
#pragma unroll
    for (int t = 0; t < kTopQPT; ++t) s1[t] = s2[t] = 0.f;
    for (int k4 = 0; k4 < D / 4; ++k4) {
      const float4 v4 = reinterpret_cast<const float4*>(Vs + ti * LD)[k4];
      const float vk[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float4 qa = reinterpret_cast<const float4*>(Lqt + (4 * k4 + c) * kTopQ + jb)[0];
        s1[0] = fmaf(vk[c], qa.x, s1[0]); s1[1] = fmaf(vk[c], qa.y, s1[1]);
        s1[2] = fmaf(vk[c], qa.z, s1[2]); s1[3] = fmaf(vk[c], qa.w, s1[3]);
      }
      if (symmetric) {
        const float4 l4 = reinterpret_cast<const float4*>(Ls + ti * LD)[k4];
        const float lk[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 ra = reinterpret_cast<const float4*>(Rqt + (4 * k4 + c) * kTopQ + jb)[0];
          s2[0] = fmaf(lk[c], ra.x, s2[0]); s2[1] = fmaf(lk[c], ra.y, s2[1]);
          s2[2] = fmaf(lk[c], ra.z, s2[2]); s2[3] = fmaf(lk[c], ra.w, s2[3]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kTopQPT; ++t) S[ti * (kTopQ + 1) + jb + t] = symmetric ? fmaxf(s1[t], s2[t]) : s1[t];
    __syncthreads();
    // merge: warp w owns queries w, w + 8, ...; lane l holds slab rows l and l + 32
    for (int j = warp; j < nq; j += kTopThreads / 32) {
      unsigned long long* L = lists + j * K;
      const int u = qs[j];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int i = lane + 32 * half;
        const long long v = v0 + i;
        const bool real = v < n && v != u && u >= 0;
        const unsigned long long key = real ? topk_key(S[i * (kTopQ + 1) + j], (int)v) : 0ull;
        unsigned want = __ballot_sync(0xffffffffu, key > L[K - 1]);
        while (want) {   // insert the candidates one by one, in lane order
          const int src = __ffs(want) - 1;
          want &= want - 1;
          const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
          if (kk <= L[K - 1]) continue;   // every lane reads the same entry: uniform
          // position = number of entries above kk; the entries from there on move down one
          int pos = 0;
          unsigned long long mine[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int e = lane + 32 * c;
            mine[c] = e < K ? L[e] : 0ull;
            pos += __popc(__ballot_sync(0xffffffffu, e < K && mine[c] > kk));
          }
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int e = lane + 32 * c;
            if (e < K - 1 && e >= pos) L[e + 1] = mine[c];
          }
          __syncwarp();
          if (lane == 0) L[pos] = kk;
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < nq * K; i += kTopThreads) part[(size_t)blockIdx.x * kTopQ * K + i] = lists[i];
}

// One CTA per query: bitonic sort (decreasing) of the nparts x K keys, first K written out.
__global__ void __launch_bounds__(kMergeThreads) k_topk_merge(const unsigned long long* __restrict__ part, int nparts,
                                                              int K, int P2, int32_t* out_idx, float* out_score) {
  extern __shared__ unsigned long long keys[];
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < P2; i += kMergeThreads) {
    unsigned long long k = 0ull;
    if (i < nparts * K) {
      const int p = i / K, e = i % K;
      k = part[(size_t)p * kTopQ * K + (size_t)j * K + e];
    }
    keys[i] = k;
  }
  __syncthreads();
  for (int size = 2; size <= P2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P2; i += kMergeThreads) {
        const int o = i ^ stride;
        if (o > i) {
          const bool desc = (i & size) == 0;
          const unsigned long long a = keys[i], b = keys[o];
          if (desc ? (a < b) : (a > b)) {
            keys[i] = b;
            keys[o] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < K; e += kMergeThreads) {
    const unsigned long long k = keys[e];
    out_idx[(size_t)j * K + e] = k ? key_id(k) : -1;
    out_score[(size_t)j * K + e] = k ? key_score(k) : __int_as_float(0xff800000);
  }
}

template <int D>
static cudaError_t pairs_impl(Ctx* c, const int32_t* src, const int32_t* dst, int count, const float* base,
                              const float* pre, int symmetric, float* scores, int sms, cudaStream_t s) {
  constexpr int RPW = 32 / (D / 4);
  const size_t sm = (size_t)D * D * sizeof(float);
  cudaFuncSetAttribute(k_score_pairs<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  long long blocks = ((long long)count + 8 * RPW - 1) / (8 * RPW);
  if (blocks > 4ll * sms) blocks = 4ll * sms;
  k_score_pairs<D><<<(int)blocks, 256, sm, s>>>(src, dst, count, c->n, c->hdr, c->ws.sG, base, pre, c->Vb,
                                                symmetric, scores);
  return cudaGetLastError();
}

template <int D>
static cudaError_t topk_impl(Ctx* c, const int32_t* rows, int count, int K, const float* base, const float* pre,
                             int symmetric, int32_t* out_idx, float* out_score, int sms, cudaStream_t s) {
  const long long nslab = ((long long)c->n + kTopSlab - 1) / kTopSlab;
  long long grid = sms;
  if (grid > kTopMaxCtas) grid = kTopMaxCtas;
  if (grid > kMergeKeys / K) grid = kMergeKeys / K;
  if (grid > nslab) grid = nslab;
  if (grid < 1) grid = 1;
  const int sym = symmetric ? 2 : 1;
  const size_t scan_sm = (size_t)kTopQ * K * 8 + (size_t)sym * kTopSlab * (D + 4) * 4 + (size_t)sym * D * kTopQ * 4 +
                         (size_t)kTopSlab * (kTopQ + 1) * 4;
  int P2 = 2;
  while (P2 < grid * K) P2 <<= 1;
  cudaFuncSetAttribute(k_topk_scan<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scan_sm);
  cudaFuncSetAttribute(k_topk_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, P2 * 8);
  for (int q0 = 0; q0 < count; q0 += kTopQ) {
    const int nq = count - q0 < kTopQ ? count - q0 : kTopQ;
    k_topk_queries<D><<<nq, 128, 0, s>>>(rows + q0, nq, c->n, c->hdr, c->ws.sG, base, pre, c->Vb, c->ws.sLq,
                                         c->ws.sRq, c->ws.sQid);
    k_topk_scan<D><<<(int)grid, kTopThreads, scan_sm, s>>>(nq, c->n, K, c->ws.sQid, c->ws.sLq, c->ws.sRq, base, pre,
                                                           c->Vb, symmetric, c->ws.sPart);
    k_topk_merge<<<nq, kMergeThreads, (size_t)P2 * 8, s>>>(c->ws.sPart, (int)grid, K, P2, out_idx + (size_t)q0 * K,
                                                          out_score + (size_t)q0 * K);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c->launches += 3;
  }
  return cudaSuccess;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

#define DAMF_SCORE_DISPATCH(fn, ...)                 \
  switch (c->d) {                                   \
    case 16: return fn<16>(c, __VA_ARGS__);          \
    case 32: return fn<32>(c, __VA_ARGS__);          \
    case 64: return fn<64>(c, __VA_ARGS__);          \
    default: return fn<128>(c, __VA_ARGS__);         \
  }

cudaError_t launch_score_pairs(Ctx* c, const int32_t* src, const int32_t* dst, int count, int context, int symmetric,
                               float* scores, cudaStream_t s) {
  k_score_prep<<<1, 1024, 0, s>>>(c->PU, c->PV, c->sigma, c->s0, c->ws.sG, c->ws.sIs0, c->d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || count == 0) return e;
  c->launches += 2;
  const float* base = context == 0 ? c->Zb : c->Ub;
  const float* pre = context == 0 ? c->ws.sIs0 : nullptr;
  const int sms = sm_count();
  DAMF_SCORE_DISPATCH(pairs_impl, src, dst, count, base, pre, symmetric, scores, sms, s)
}

cudaError_t launch_topk(Ctx* c, const int32_t* rows, int count, int k, int context, int symmetric, int32_t* out_idx,
                        float* out_score, cudaStream_t s) {
  k_score_prep<<<1, 1024, 0, s>>>(c->PU, c->PV, c->sigma, c->s0, c->ws.sG, c->ws.sIs0, c->d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || count == 0) return e;
  c->launches += 1;
  const float* base = context == 0 ? c->Zb : c->Ub;
  const float* pre = context == 0 ? c->ws.sIs0 : nullptr;
  const int sms = sm_count();
  DAMF_SCORE_DISPATCH(topk_impl, rows, count, k, base, pre, symmetric, out_idx, out_score, sms, s)
}

}  // namespace damf
