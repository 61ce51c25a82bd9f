// Dynamic embedding enhancement (Sec. 4.4; Step 4 of Sec. 4.5): PPR push rounds.
//
// State (Zb, r) keeps  Pi X_b = Zb + Pi r  with P = D^{-1} A, Pi = alpha (I - (1-alpha) P)^{-1}.
// Because Pi = alpha I + (1-alpha) Pi P, pushing node u moves alpha r[u] into Zb[u] and
// adds (1-alpha) A[w][u] / deg(w) * r[u] to r[w] for every in-neighbour w of u. Any order of
// pushes keeps the invariant. The push stops when no row has max_j |r[u][j]| > eps; then
// |Zb - Pi X_b| <= eps elementwise since Pi is row-substochastic. With the degree-scaled
// threshold (damf_config.threshold = 1) the eps of row u reads eps * max(deg(u), 1), deg the
// out-degree, and the bound becomes |Zb - Pi X_b|[i] <= (Pi t)[i] for those thresholds t.
//
// One persistent cooperative launch runs all rounds, with one bounded grid barrier per round.
// Round k works on
//   - the candidates queued for it (rows whose residual may exceed eps). A row group reads
//     v = r[u]; if max|v| > eps it removes exactly v with a float4 atomic add of -v (adds of
//     other pushes of the same round may land before or after it; both stay accounted for),
//     adds alpha v to Zb[u], and scatters coef * v to the in-neighbours of u itself when u
//     has few in-edges. For more, v goes to a rho slot and u's in-edges are cut into work
//     items for round k+1, which spreads a hub's in-edges over every warp;
//   - the work items that round k-1 deferred to it.
// Every atomic add returns the old value, so the thread whose add (or removal) is the last
// one on an element sees the value the round leaves there; a row left above eps is queued
// once (per-round stamp) for round k+1. When round k queues no row and no item, no row
// exceeds eps.
// Lists and rho are double-buffered by round parity; their counters are indexed by round
// mod 3, so block 0 resets the counters of round k+2 while those of rounds k and k+1 are
// in use.
#include <stdlib.h>

#include "damf_internal.cuh"

namespace damf {

// CTAs of the push per SM: leaves registers, threads and shared memory on every SM for
// the one-CTA kernels of the next update's factor chain (overridable for tuning with the
// environment variable DAMF_PUSH_CTAS_PER_SM).
constexpr int kPushBlocksPerSM = 2;
// A pushing row group scatters to at most this many chunks of in-edges itself; rows with
// more in-edges are deferred as work items (overridable with DAMF_PUSH_DIRECT_CHUNKS).
constexpr int kPushDirectChunks = 1;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// adds the time since the last mark to slot i and sets a new mark
__device__ __forceinline__ void time_mark(unsigned long long* s_t, int i) {
  const unsigned long long t = gtimer();
  s_t[i] += t - s_t[4];
  s_t[4] = t;
}

__device__ __forceinline__ float4 f4_ldcg(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ float max_abs4(float4 v) {
  return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
}

// in-edges per chunk: one per lane of a row group, at most 8
template <int D>
struct PushShape {
  static constexpr int LPR = D / 4;                 // lanes per row (float4 each)
  static constexpr int RPW = 32 / LPR;              // row groups per warp
  static constexpr int CH = LPR < 8 ? LPR : 8;      // in-edges per chunk
};

// maximum over the LPR lanes of a row group (every lane of the warp takes part)
template <int LPR>
__device__ __forceinline__ float group_max(float m) {
#pragma unroll
  for (int o = 1; o < LPR; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// queues w for the next round unless this round already has
__device__ __forceinline__ void enqueue(int w, unsigned tag, uint32_t* stamp, int* count, int32_t* list) {
  if (atomicExch(stamp + w, tag) != tag) {
    const int p = atomicAdd(count, 1);
    __stcg(list + p, w);
  }
}

// Threshold of a node with out-degree deg: eps, or eps * max(deg, 1) when SCALED.
template <bool SCALED>
__device__ __forceinline__ float threshold(float eps, int deg) {
  return SCALED ? eps * (float)max(deg, 1) : eps;
}

// One chunk of a scatter by a row group: lane q < ne owns in-edge col[st + q] (node w) and
// its coefficient (1-alpha)/deg(w); every lane adds coef * rv to its float4 of r[w] for each
// of the ne in-edges, all atomics in flight before any result is looked at. A w that an add
// left above its threshold is queued for the next round. Every lane of the warp calls this;
// a group with nothing to do passes ne = 0.
template <int D, bool SCALED>
__device__ __forceinline__ void scatter_chunk(const float4 rv, int st, int ne, const int32_t* __restrict__ col,
                                              const int32_t* __restrict__ outdeg, float* r, float beta, float eps,
                                              unsigned tag, uint32_t* stamp, int* next_count, int32_t* next_list,
                                              int q, int sub, unsigned sub_mask) {
  constexpr int LPR = PushShape<D>::LPR;
  constexpr int CH = PushShape<D>::CH;
  int w_own = 0, d_own = 1;
  float c_own = 0.f;
  if (q < ne) {
    w_own = __ldg(col + st + q);
    d_own = __ldg(outdeg + w_own);
    c_own = beta / (float)d_own;
  }
  float4 nv[CH];
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    const int w = __shfl_sync(0xffffffffu, w_own, sub * LPR + e);
    const float coef = __shfl_sync(0xffffffffu, c_own, sub * LPR + e);
    nv[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < ne) {
      const float4 add = make_float4(coef * rv.x, coef * rv.y, coef * rv.z, coef * rv.w);
      const float4 old = atomicAdd(reinterpret_cast<float4*>(r + (size_t)w * D) + q, add);
      nv[e] = make_float4(old.x + add.x, old.y + add.y, old.z + add.z, old.w + add.w);
    }
  }
  unsigned crossed_bits = 0;
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    const float thr = SCALED ? __shfl_sync(0xffffffffu, threshold<true>(eps, d_own), sub * LPR + e) : eps;
    if (__ballot_sync(0xffffffffu, max_abs4(nv[e]) > thr) & sub_mask) crossed_bits |= 1u << e;
  }
  if (q < ne && ((crossed_bits >> q) & 1u)) enqueue(w_own, tag, stamp, next_count, next_list);
}

// 64 registers at most (min. 4 CTAs' worth per SM): two push CTAs (32k registers) then leave room
// on every SM for the 768-thread core SVD CTA of the next update, which runs beside the push
template <int D, bool SCALED>
__global__ void __launch_bounds__(256, 4) k_push(DevHeader* h, Adj in, const int32_t* __restrict__ outdeg, Workspace ws,
                                                 float* Zb, float* r, int n, float alpha, float eps, int max_rounds,
                                                 int check_all, int direct_max) {
  constexpr int LPR = PushShape<D>::LPR;
  constexpr int RPW = PushShape<D>::RPW;
  constexpr int CH = PushShape<D>::CH;
  const unsigned nblocks = gridDim.x;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR, q = lane % LPR;
  const unsigned sub_mask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << (sub * LPR));
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned epoch0 = h->epoch;
  const float beta = 1.0f - alpha;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  long long my_pushes = 0, my_edges = 0;
  const int ncand0 = check_all ? n : h->pending;
  // block 0's view of where the time goes (ns): deferred items, candidates, barrier;
  // [4] is the last time mark. Kept in shared memory, where it costs no registers.
  __shared__ unsigned long long s_t[5];
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  if (timer) s_t[0] = s_t[1] = s_t[2] = s_t[3] = 0ull;
  int round = 0;
  for (;;) {
    if (round >= max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(h, DAMF_ERR_NOT_CONVERGED);
      break;
    }
    if (timer) s_t[4] = gtimer();
    const int P = round & 1;
    const int K0 = round % 3, K1 = (round + 1) % 3, K2 = (round + 2) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // last read in round k-1, next written in round k+1
      h->cand_count[K2] = 0;
      h->front_count[K2] = 0;
      h->work_count[K2] = 0;
    }
    const unsigned tag = epoch0 + (unsigned)round + 1u;
    int* next_count = &h->cand_count[K1];
    int32_t* next_list = ws.cand[P ^ 1];

    // ---- work items deferred by the previous round ----
    const int nwork = round == 0 ? 0 : __ldcg(&h->work_count[K0]);
    const float* rho_in = ws.rho[P];
    const int4* work_in = ws.work[P];
    for (long long it = gwarp * RPW + sub; it - sub < nwork; it += nwarps * RPW) {
      int4 wi = make_int4(0, 0, 0, 0);
      float4 rv = zero4;
      if (it < nwork) {
        wi = __ldcg(work_in + it);
        rv = f4_ldcg(rho_in + (size_t)wi.x * D + 4 * q);
      }
      scatter_chunk<D, SCALED>(rv, wi.y, wi.z, in.col, outdeg, r, beta, eps, tag, ws.stamp, next_count, next_list, q, sub,
                       sub_mask);
    }
    if (timer) time_mark(s_t, 0);

    // ---- candidates ----
    const int ncand = round == 0 ? ncand0 : __ldcg(&h->cand_count[K0]);
    const int32_t* cand = round == 0 ? (check_all ? nullptr : ws.pend) : ws.cand[P];
    float* rho_out = ws.rho[P ^ 1];
    int4* work_out = ws.work[P ^ 1];
    for (long long base = gwarp * RPW; base < ncand; base += nwarps * RPW) {
      const long long ci = base + sub;
      const bool valid = ci < ncand;
      const int u = valid ? (cand ? __ldcg(cand + ci) : (int)ci) : 0;
      float4 v = zero4, z = zero4;
      int st = 0, deg = 0, dout = 1;
      if (valid) {   // everything that depends only on u is requested at once
        v = f4_ldcg(r + (size_t)u * D + 4 * q);
        z = f4_ldcg(Zb + (size_t)u * D + 4 * q);
        st = in.start[u];
        deg = in.len[u];
        if (SCALED) dout = __ldg(outdeg + u);
      }
      const float thr_u = threshold<SCALED>(eps, dout);
      const bool push = group_max<LPR>(max_abs4(v)) > thr_u && valid;
      float lm = 0.f;   // max |r[u]| right after the removal of v (over this lane's float4)
      if (push) {
        const float4 old =
            atomicAdd(reinterpret_cast<float4*>(r + (size_t)u * D) + q, make_float4(-v.x, -v.y, -v.z, -v.w));
        lm = max_abs4(make_float4(old.x - v.x, old.y - v.y, old.z - v.z, old.w - v.w));
        z.x = fmaf(alpha, v.x, z.x);
        z.y = fmaf(alpha, v.y, z.y);
        z.z = fmaf(alpha, v.z, z.z);
        z.w = fmaf(alpha, v.w, z.w);
        __stcg(reinterpret_cast<float4*>(Zb + (size_t)u * D) + q, z);
        if (q == 0) {
          my_pushes += 1;
          my_edges += deg;
        }
      }
      // many in-edges: a rho slot and work items for the next round (warp-aggregated slots)
      const bool defer = push && deg > direct_max;
      const unsigned bal = __ballot_sync(0xffffffffu, defer && q == 0);
      if (bal) {
        const int nch = defer ? (deg + CH - 1) / CH : 0;
        int wsum = (q == 0) ? nch : 0, wpre = wsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {   // inclusive prefix sum over the warp
          const int t = __shfl_up_sync(0xffffffffu, wpre, o);
          if (lane >= o) wpre += t;
        }
        const int wtot = __shfl_sync(0xffffffffu, wpre, 31);
        int basepos = 0, wbase = 0;
        if (lane == 0) {
          basepos = atomicAdd(&h->front_count[K1], __popc(bal));
          wbase = atomicAdd(&h->work_count[K1], wtot);
        }
        basepos = __shfl_sync(0xffffffffu, basepos, 0);
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        const int wmine = __shfl_sync(0xffffffffu, wpre - wsum, sub * LPR);   // exclusive prefix of my group
        if (defer) {
          const int pos = basepos + __popc(bal & ((1u << (sub * LPR)) - 1u));
          __stcg(reinterpret_cast<float4*>(rho_out + (size_t)pos * D) + q, v);
          for (int c2 = q; c2 < nch; c2 += LPR) {
            const int e0 = c2 * CH;
            __stcg(work_out + wbase + wmine + c2, make_int4(pos, st + e0, min(CH, deg - e0), 0));
          }
        }
      }
      // few in-edges: scatter now, one chunk of CH in-edges per step (warp-uniform trip count)
      const int ndir = (push && !defer) ? (deg + CH - 1) / CH : 0;
      int nmax = ndir;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
      for (int c2 = 0; c2 < nmax; ++c2) {
        const int e0 = c2 * CH;
        const int ne = c2 < ndir ? min(CH, deg - e0) : 0;
        scatter_chunk<D, SCALED>(v, st + e0, ne, in.col, outdeg, r, beta, eps, tag, ws.stamp, next_count, next_list, q, sub,
                         sub_mask);
      }
      // u itself: adds that reached r[u] between the read of v and its removal are still there
      lm = group_max<LPR>(lm);
      if (push && q == 0 && lm > thr_u) enqueue(u, tag, ws.stamp, next_count, next_list);
    }
    if (timer) time_mark(s_t, 1);
    if (!grid_barrier(&h->bar, h, nblocks)) return;
    if (timer) time_mark(s_t, 2);
    ++round;
    if (__ldcg(&h->cand_count[K1]) == 0 && __ldcg(&h->work_count[K1]) == 0) break;
  }
  if (timer)
    for (int i = 0; i < 4; ++i) h->push_ns[i] += s_t[i];
  // counters and bookkeeping (block 0 after the last barrier; everyone has left the loop)
  for (int o = 16; o > 0; o >>= 1) {
    my_pushes += __shfl_xor_sync(0xffffffffu, my_pushes, o);
    my_edges += __shfl_xor_sync(0xffffffffu, my_edges, o);
  }
  if (lane == 0 && (my_pushes || my_edges)) {
    atomicAdd((unsigned long long*)&h->pushes, (unsigned long long)my_pushes);
    atomicAdd((unsigned long long*)&h->push_edges, (unsigned long long)my_edges);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    h->push_rounds += round;
    h->pending = 0;
    h->check_all = 0;
    h->epoch = epoch0 + (unsigned)round + 2u;
  }
}

template <int D, bool SCALED>
static cudaError_t push_impl(Ctx* c, int check_all, cudaStream_t s) {
  if (c->push_blocks == 0) {
    // two CTAs per SM: leaves registers, threads and shared memory on every SM for the
    // one-CTA kernels of the next update's factor chain, which overlap the push
    cudaFuncSetAttribute(k_push<D, SCALED>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<D, SCALED>, 256, 0);
    int cap = kPushBlocksPerSM;
    if (const char* ev = getenv("DAMF_PUSH_CTAS_PER_SM")) {
      const int v = atoi(ev);
      if (v >= 1 && v <= 8) cap = v;
    }
    if (per_sm > cap) per_sm = cap;
    c->push_blocks = sms * (per_sm < 1 ? 1 : per_sm);
  }
  int chunks = kPushDirectChunks;
  if (const char* ev = getenv("DAMF_PUSH_DIRECT_CHUNKS")) {
    const int v = atoi(ev);
    if (v >= 0 && v <= 64) chunks = v;
  }
  cudaError_t e = cudaMemsetAsync(&c->hdr->cand_count[0], 0, 9 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  DevHeader* h = c->hdr;
  Adj in = c->cfg.directed ? c->in : c->out;
  const int32_t* outdeg = c->out.len;
  Workspace ws = c->ws;
  float* Zb = c->Zb;
  float* r = c->r;
  int n = c->n;
  float alpha = (float)c->cfg.alpha, eps = (float)c->cfg.eps;
  int max_rounds = c->cfg.max_push_rounds;
  int direct_max = chunks * PushShape<D>::CH;
  void* args[] = {&h, &in, &outdeg, &ws, &Zb, &r, &n, &alpha, &eps, &max_rounds, &check_all, &direct_max};
  return cudaLaunchCooperativeKernel((void*)k_push<D, SCALED>, dim3(c->push_blocks), dim3(256), args, 0, s);
}

template <bool SCALED>
static cudaError_t push_dispatch(Ctx* c, int check_all, cudaStream_t s) {
  switch (c->d) {
    case 16: return push_impl<16, SCALED>(c, check_all, s);
    case 32: return push_impl<32, SCALED>(c, check_all, s);
    case 64: return push_impl<64, SCALED>(c, check_all, s);
    default: return push_impl<128, SCALED>(c, check_all, s);
  }
}

cudaError_t launch_push(Ctx* c, int check_all, cudaStream_t s) {
  return c->cfg.threshold ? push_dispatch<true>(c, check_all, s) : push_dispatch<false>(c, check_all, s);
}

}  // namespace damf
