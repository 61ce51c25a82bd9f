// Dynamic embedding enhancement (Sec. 4.4; Step 4 of Sec. 4.5): PPR push rounds.
//
// State (Zb, r) keeps  Pi X_b = Zb + Pi r  with P = D^{-1} A, Pi = alpha (I - (1-alpha) P)^{-1}.
// Because Pi = alpha I + (1-alpha) Pi P, pushing node u moves alpha r[u] into Zb[u] and
// adds (1-alpha) A[w][u] / deg(w) * r[u] to r[w] for every in-neighbour w of u.
// Rounds: the frontier is {u : max_j |r[u][j]| > eps} among the candidates (rows whose
// residual may have crossed eps).  When no row exceeds eps, |Zb - Pi X_b| <= eps
// elementwise since Pi is row-substochastic.
//
// One persistent cooperative launch runs all rounds; two bounded grid barriers per round:
//   phase A: candidates -> frontier rows; rho[pos] = r[u], r[u] = 0, Zb[u] += alpha rho,
//            and the in-edges of u cut into work items (one in-edge per lane of a row group);
//   phase B: each work item adds coef * rho to r[w] with float4 atomics (L2), all of an
//            item's atomics in flight at once; a row whose new value crosses eps is
//            queued once per round (stamp) as a candidate.
// Counters are indexed by round parity so each is reset by one block between its uses.
#include <stdlib.h>

#include "damf_internal.cuh"

namespace damf {

// CTAs of the push per SM: leaves registers, threads and shared memory on every SM for
// the one-CTA kernels of the next update's factor chain (overridable for tuning with the
// environment variable DAMF_PUSH_CTAS_PER_SM).
constexpr int kPushBlocksPerSM = 2;

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

// in-edges per work item: one per lane of a row group, at most 8
template <int D>
struct PushShape {
  static constexpr int LPR = D / 4;                 // lanes per row (float4 each)
  static constexpr int RPW = 32 / LPR;              // row groups per warp
  static constexpr int CH = LPR < 8 ? LPR : 8;      // in-edges per work item
};

// 64 registers at most (min. 4 CTAs' worth per SM): two push CTAs (32k registers) then leave room
// on every SM for the 768-thread core SVD CTA of the next update, which runs beside the push
template <int D>
__global__ void __launch_bounds__(256, 4) k_push(DevHeader* h, Adj in, const int32_t* __restrict__ outdeg, Workspace ws,
                                              float* Zb, float* r, int n, float alpha, float eps, int max_rounds,
                                              int check_all) {
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
  long long my_pushes = 0, my_edges = 0;
  const int ncand0 = check_all ? n : h->pending;
  int round = 0;
  // block 0's view of where the time goes (ns): phase A, barrier after A, phase B, barrier after B;
  // [4] is the last time mark. Kept in shared memory, where it costs no registers.
  __shared__ unsigned long long s_t[5];
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  if (timer) s_t[0] = s_t[1] = s_t[2] = s_t[3] = 0ull;
  for (;; ++round) {
    if (timer) s_t[4] = gtimer();
    const int P = round & 1;
    if (round >= max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(h, DAMF_ERR_NOT_CONVERGED);
      break;
    }
    // ---- phase A: frontier ----
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      h->front_count[P ^ 1] = 0;
      h->work_count[P ^ 1] = 0;
    }
    const int ncand = round == 0 ? ncand0 : __ldcg(&h->cand_count[P]);
    const int32_t* cand = round == 0 ? (check_all ? nullptr : ws.pend) : ws.cand[P];
    for (long long base = gwarp * RPW; base < ncand; base += nwarps * RPW) {
      const long long ci = base + sub;
      const bool valid = ci < ncand;
      const int u = valid ? (cand ? __ldcg(cand + ci) : (int)ci) : 0;
      // everything that depends only on u is requested at once
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f), z = v;
      int st = 0, deg = 0;
      if (valid) {
        v = f4_ldcg(r + (size_t)u * D + 4 * q);
        z = f4_ldcg(Zb + (size_t)u * D + 4 * q);
        st = in.start[u];
        deg = in.len[u];
      }
      float mx = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const bool push = valid && mx > eps;
      const int nch = push ? (deg + CH - 1) / CH : 0;
      // warp-aggregated slots: one frontier row per pushing group, nch work items each
      const unsigned bal = __ballot_sync(0xffffffffu, push && q == 0);
      int wsum = (q == 0) ? nch : 0, wpre = wsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {   // inclusive prefix sum over the warp
        const int t = __shfl_up_sync(0xffffffffu, wpre, o);
        if (lane >= o) wpre += t;
      }
      const int wtot = __shfl_sync(0xffffffffu, wpre, 31);
      int basepos = 0, wbase = 0;
      if (lane == 0 && bal) {
        basepos = atomicAdd(&h->front_count[P], __popc(bal));
        if (wtot) wbase = atomicAdd(&h->work_count[P], wtot);
      }
      basepos = __shfl_sync(0xffffffffu, basepos, 0);
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      const int wmine = __shfl_sync(0xffffffffu, wpre - wsum, sub * LPR);   // exclusive prefix of my group
      if (push) {
        const int pos = basepos + __popc(bal & ((1u << (sub * LPR)) - 1u));
        __stcg(reinterpret_cast<float4*>(ws.rho + (size_t)pos * D) + q, v);
        __stcg(reinterpret_cast<float4*>(r + (size_t)u * D) + q, make_float4(0.f, 0.f, 0.f, 0.f));
        z.x = fmaf(alpha, v.x, z.x);
        z.y = fmaf(alpha, v.y, z.y);
        z.z = fmaf(alpha, v.z, z.z);
        z.w = fmaf(alpha, v.w, z.w);
        __stcg(reinterpret_cast<float4*>(Zb + (size_t)u * D) + q, z);
        // work item: (rho slot, first in-edge, number of in-edges)
        for (int c2 = q; c2 < nch; c2 += LPR) {
          const int e0 = c2 * CH;
          __stcg(&ws.work[wbase + wmine + c2], make_int4(pos, st + e0, min(CH, deg - e0), 0));
        }
        if (q == 0) {
          my_pushes += 1;
          my_edges += deg;
        }
      }
    }
    if (timer) time_mark(s_t, 0);
    if (!grid_barrier(&h->bar, h, nblocks)) return;
    if (timer) time_mark(s_t, 1);
    const int nfront = __ldcg(&h->front_count[P]);
    if (nfront == 0) break;
    // ---- phase B: scatter (1-alpha) rho / deg(w) to in-neighbours ----
    if (blockIdx.x == 0 && threadIdx.x == 0) h->cand_count[P] = 0;
    const int nwork = __ldcg(&h->work_count[P]);
    const unsigned tag = epoch0 + (unsigned)round + 1u;
    for (long long it = gwarp * RPW + sub; it - sub < nwork; it += nwarps * RPW) {
      const bool valid = it < nwork;
      int4 wi = make_int4(0, 0, 0, 0);
      if (valid) wi = __ldcg(&ws.work[it]);
      const int ne = wi.z;
      // lane q < ne of the row group owns in-edge wi.y + q; rho is requested alongside
      int w_own = 0;
      if (q < ne) w_own = __ldg(in.col + wi.y + q);
      float4 rv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) rv = f4_ldcg(ws.rho + (size_t)wi.x * D + 4 * q);
      float c_own = 0.f;
      if (q < ne) c_own = beta / (float)__ldg(outdeg + w_own);
      // issue every atomic of the item before looking at any result
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
        const bool cr = fmaxf(fmaxf(fabsf(nv[e].x), fabsf(nv[e].y)), fmaxf(fabsf(nv[e].z), fabsf(nv[e].w))) > eps;
        if (__ballot_sync(0xffffffffu, cr) & sub_mask) crossed_bits |= 1u << e;
      }
      // lane q handles the stamp of its own edge
      if (q < ne && ((crossed_bits >> q) & 1u)) {
        if (atomicExch(&ws.stamp[w_own], tag) != tag) {
          const int p = atomicAdd(&h->cand_count[P ^ 1], 1);
          __stcg(ws.cand[P ^ 1] + p, w_own);
        }
      }
    }
    if (timer) time_mark(s_t, 2);
    if (!grid_barrier(&h->bar, h, nblocks)) return;
    if (timer) time_mark(s_t, 3);
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

template <int D>
static cudaError_t push_impl(Ctx* c, int check_all, cudaStream_t s) {
  if (c->push_blocks == 0) {
    // two CTAs per SM: leaves registers, threads and shared memory on every SM for the
    // one-CTA kernels of the next update's factor chain, which overlap the push
    cudaFuncSetAttribute(k_push<D>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<D>, 256, 0);
    int cap = kPushBlocksPerSM;
    if (const char* ev = getenv("DAMF_PUSH_CTAS_PER_SM")) {
      const int v = atoi(ev);
      if (v >= 1 && v <= 8) cap = v;
    }
    if (per_sm > cap) per_sm = cap;
    c->push_blocks = sms * (per_sm < 1 ? 1 : per_sm);
  }
  cudaError_t e = cudaMemsetAsync(&c->hdr->cand_count[0], 0, 6 * sizeof(int), s);
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
  void* args[] = {&h, &in, &outdeg, &ws, &Zb, &r, &n, &alpha, &eps, &max_rounds, &check_all};
  return cudaLaunchCooperativeKernel((void*)k_push<D>, dim3(c->push_blocks), dim3(256), args, 0, s);
}

cudaError_t launch_push(Ctx* c, int check_all, cudaStream_t s) {
  switch (c->d) {
    case 16: return push_impl<16>(c, check_all, s);
    case 32: return push_impl<32>(c, check_all, s);
    case 64: return push_impl<64>(c, check_all, s);
    default: return push_impl<128>(c, check_all, s);
  }
}

}  // namespace damf
