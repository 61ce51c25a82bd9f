// Rediagonalisation (Step 2 of Sec. 4.5; Eq. "svd_small_edge"): the top-d SVD of the
// (d + r) x (d + r) core M by one-sided (Hestenes) Jacobi on a cluster of kClP CTAs.
//
// One-sided Jacobi orthogonalises the columns of A = M J by plane rotations; at convergence
// the columns are U Theta. Here the columns are cut into kClBlocks = 2 kClP blocks of bs
// columns and each CTA holds two blocks in shared memory. A sweep is kClBlocks - 1 steps of
// a circle-method tournament over the blocks: in step t CTA c holds a pair of blocks and
// rotates every column pair between them (in step 0 also every pair inside them, which
// covers the pairs within each block once per sweep); between steps the CTAs pull the blocks
// of the next step from each other's shared memory (distributed shared memory, one cluster
// barrier: the two buffers alternate). Every column pair is visited once per sweep, as in the one-CTA order, while
// each CTA works on an eighth of the columns: eight SMs issue the rotations instead of one.
// Within a step a warp rotates one pair per round (rounds of disjoint pairs separated by
// __syncthreads), holding both columns in registers between the dot product and the rotation.
// Squared norms are cached per column and travel with the blocks; they are recomputed
// exactly at the start of every sweep and shared with every CTA of the cluster.
// Only pairs with a column among the current top d (by norm) rotate; when a sweep rotates
// nothing, the top columns are orthogonal to each other and to the rest, so they are the top
// singular vectors provided no discarded column can hide a larger singular value: checked by
// the Cauchy-Schwarz bound max_j |a_j| * sum_i |a_i| (discarded columns) < min top norm^2.
// When that fails, or the top set keeps rotating after kTopOnlySweeps sweeps, every pair is
// rotated from then on. Every CTA takes these decisions from the same shared values, so all
// of them pass the same cluster barriers.
#include <cooperative_groups.h>

#include "damf_internal.cuh"

namespace cg = cooperative_groups;

namespace damf {

constexpr int kClP = 8;                          // CTAs per cluster (the portable maximum)
constexpr int kClBlocks = 2 * kClP;              // column blocks
constexpr int kClL = kClBlocks - 1;              // steps per sweep
constexpr int kClBsMax = kMaxM / kClBlocks;      // 16 columns per block at most
// 16 warps at <= 64 registers: 4 warps of 2K registers per SM sub-partition, the half of its
// 16K register file that two CTAs of the push (256 threads x 64 registers) leave free, so
// the cluster runs beside a push; one warp per pair of a round (16 pairs at most)
constexpr int kClThreads = 512;
constexpr int kClStride = 256;                   // floats per column: rows padded with zeros
constexpr float kClTol = 1e-6f;                  // rotate while |a_p . a_q| > tol |a_p| |a_q|
constexpr int kClTopOnlySweeps = 6;
// An update's core stops after a sweep in which every rotation was small: relative coupling
// |a_p . a_q| / |a_p||a_q| and rotation tangent both below kClStopRel. The pairs it left are
// then coupled at about the product of those, and the first-order correction that follows
// (T = E^T M H) removes what remains between the top columns. (With the coupling alone as the
// measure, a cluster of nearly equal norms, whose pairs turn by large angles at any coupling,
// stopped early on a C3 core and left two columns of U coupled at 1.3e-3.)
constexpr float kClStopRel = 3e-4f;

// shared memory: columns [2 buffers][2 slots][kClBsMax][kClStride], their squared norms
// [2][2][kClBsMax], all norms by global column [kClBlocks * kClBsMax], top flags, sweep flags
constexpr size_t kClColFloats = (size_t)2 * 2 * kClBsMax * kClStride;
constexpr size_t kClSmemBytes =
    (kClColFloats + 2 * 2 * kClBsMax + kClBlocks * kClBsMax) * sizeof(float) + kClBlocks * kClBsMax + 64;

// Block held in `slot` by CTA c at step t (circle method over kClBlocks blocks, block kClL fixed).
__device__ __forceinline__ int cl_block(int c, int slot, int t) {
  if (c == 0) return slot == 0 ? kClL : t;
  return slot == 0 ? (t + c) % kClL : (t - c + kClL) % kClL;
}

// CTA and slot that hold block b at step t.
__device__ __forceinline__ void cl_holder(int b, int t, int& hc, int& hs) {
  hc = 0;
  hs = 0;
  if (b == kClL) return;
  if (b == t) {
    hs = 1;
    return;
  }
  for (int k = 1; k < kClP; ++k) {
    if ((t + k) % kClL == b) {
      hc = k;
      return;
    }
    if ((t - k + kClL) % kClL == b) {
      hc = k;
      hs = 1;
      return;
    }
  }
}

// Circle-method pairing of nl (even) items: round t, pair k.
__device__ __forceinline__ void cl_pair(int nl, int round, int k, int& p, int& q) {
  const int L = nl - 1;
  if (k == 0) {
    p = L;
    q = round;
  } else {
    p = round + k;
    p -= p >= L ? L : 0;
    q = round - k + L;
    q -= q >= L ? L : 0;
  }
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// One pair (warp-level): columns ap, aq of kClStride floats (lane holds rows 4 lane .. +3 and,
// when TWO, 128 + 4 lane .. +3), cached squared norms np, nq. Rotates when
// |g| > tol |a_p||a_q| (the rotation makes the two columns orthogonal); returns whether it did.
template <bool TWO>
__device__ __forceinline__ bool cl_rotate(float* ap, float* aq, float* np, float* nq, int lane, float tol2,
                                          float& rel2) {
  float4* p4 = reinterpret_cast<float4*>(ap) + lane;
  float4* q4 = reinterpret_cast<float4*>(aq) + lane;
  const float4 x0 = p4[0], y0 = q4[0];
  const float4 x1 = TWO ? p4[32] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 y1 = TWO ? q4[32] : make_float4(0.f, 0.f, 0.f, 0.f);
  float2 acc = __fmul2_rn(lo2(x0), lo2(y0));
  acc = __ffma2_rn(hi2(x0), hi2(y0), acc);
  if (TWO) {
    acc = __ffma2_rn(lo2(x1), lo2(y1), acc);
    acc = __ffma2_rn(hi2(x1), hi2(y1), acc);
  }
  const float g = warp_sum(acc.x + acc.y);
  const float aa = *np, bb = *nq;
  if (!(g * g > tol2 * aa * bb)) return false;
  // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / (2 g): the smaller root of
  // t^2 + 2 zeta t - 1 = 0, so that the rotated columns are orthogonal. The angle may come
  // from hardware approximations (an inexact t only leaves a smaller g for the next sweep),
  // and cs = 1/sqrt(1 + t^2) should carry no bias: the rotation scales both columns by
  // cs^2 (1 + t^2), and a column sees ~700 rotations per update. One Newton step on the
  // hardware approximation y0, y0 + (y0 / 2) (1 - x y0^2) with the residual from an FMA,
  // leaves a mean scale error of ~2e-9 per rotation (the approximation alone errs to one
  // side by ~1e-8). Singular values and vector norms no longer come from the column norms
  // (the refinement after the Newton-Schulz step normalises and takes Rayleigh quotients).
  const float zeta = __fdividef(bb - aa, 2.0f * g);
  const float az = fabsf(zeta);
  const float s1 = fmaf(az, az, 1.0f);
  const float ta = az < 1e15f ? __fdividef(1.0f, fmaf(s1, rsqrtf(s1), az)) : __fdividef(0.5f, az);
  const float t = copysignf(ta, zeta);
  const float tt1 = fmaf(t, t, 1.0f);
  const float ry = rsqrtf(tt1);
  const float dres = fmaf(-(tt1 * ry), ry, 1.0f);
  const float cs = fmaf(0.5f * ry, dres, ry);
  const float sn = cs * t;
  // the stop rule's measure: the larger of the squared relative coupling and the squared
  // rotation tangent (a pair of nearly equal norms turns by a large angle however weak its
  // coupling, and such a turn passes couplings on to the other pairs at full size)
  rel2 = fmaxf(__fdividef(g * g, aa * bb), t * t);
  const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ms2 = make_float2(-sn, -sn);
  {
    const float2 pl = __ffma2_rn(c2, lo2(x0), __fmul2_rn(ms2, lo2(y0)));
    const float2 ph = __ffma2_rn(c2, hi2(x0), __fmul2_rn(ms2, hi2(y0)));
    const float2 ql = __ffma2_rn(s2, lo2(x0), __fmul2_rn(c2, lo2(y0)));
    const float2 qh = __ffma2_rn(s2, hi2(x0), __fmul2_rn(c2, hi2(y0)));
    p4[0] = make_float4(pl.x, pl.y, ph.x, ph.y);
    q4[0] = make_float4(ql.x, ql.y, qh.x, qh.y);
  }
  if (TWO) {
    const float2 pl = __ffma2_rn(c2, lo2(x1), __fmul2_rn(ms2, lo2(y1)));
    const float2 ph = __ffma2_rn(c2, hi2(x1), __fmul2_rn(ms2, hi2(y1)));
    const float2 ql = __ffma2_rn(s2, lo2(x1), __fmul2_rn(c2, lo2(y1)));
    const float2 qh = __ffma2_rn(s2, hi2(x1), __fmul2_rn(c2, hi2(y1)));
    p4[32] = make_float4(pl.x, pl.y, ph.x, ph.y);
    q4[32] = make_float4(ql.x, ql.y, qh.x, qh.y);
  }
  if (lane == 0) {
    *np = fmaxf(aa - t * g, 0.0f);
    *nq = bb + t * g;
  }
  return true;
}

template <int D>
__global__ void __cluster_dims__(kClP, 1, 1) __launch_bounds__(kClThreads, 2)   // <= 64 registers
    k_jacobi_cl(DevHeader* h, const float* __restrict__ Min, int m_host, int use_hdr, float* E, float* theta,
                float tol, int max_sweeps) {
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  extern __shared__ __align__(16) float smem[];
  float* colbuf = smem;
  float* bnrm = colbuf + kClColFloats;
  float* allnrm = bnrm + 2 * 2 * kClBsMax;
  unsigned char* top = reinterpret_cast<unsigned char*>(allnrm + kClBlocks * kClBsMax);
  __shared__ int s_rot;
  __shared__ int s_flags[kClP];
  __shared__ unsigned s_rel2;           // largest squared relative coupling rotated in the sweep (float bits)
  __shared__ unsigned s_rels[kClP];
  // the step's pairs, round by round: (slot * kClBsMax + i) of both columns packed as p | q << 8,
  // -1 when the top-set rule leaves the pair out (built once per step, read by one warp a round)
  __shared__ int s_pairs[(2 * kClBsMax - 1) * kClBsMax];
  // the same header values for every CTA of the cluster (written by earlier kernels)
  // use_hdr: 1 = the update's core (m from the header, counters recorded), 0 = a dense
  // matrix of m_host columns, 2 = the same and non-convergence recorded as a status
  const int m = use_hdr == 1 ? D + h->nS : m_host;
  if (use_hdr == 1 && h->nS == 0) return;
  const int mp = (m + 31) & ~31;
  const int ne = mp / 32;
  const bool two = mp > 128;       // rows 128.. present: a lane holds two float4 of a column
  const int bs = (m + kClBlocks - 1) / kClBlocks;
  const int ng = kClBlocks * bs;   // global columns incl. the zero padding
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kClThreads / 32;
  const float tol2 = tol * tol;
  auto col = [&](int bf, int slot, int i) { return colbuf + ((bf * 2 + slot) * kClBsMax + i) * kClStride; };
  auto nrm = [&](int bf, int slot, int i) { return bnrm + (bf * 2 + slot) * kClBsMax + i; };

  // blocks of step 0
  for (int slot = 0; slot < 2; ++slot) {
    const int b = cl_block(c, slot, 0);
    for (int o = tid; o < bs * kClStride; o += kClThreads) {
      const int i = o / kClStride, row = o % kClStride;
      const int g = b * bs + i;
      col(0, slot, i)[row] = (g < m && row < m) ? Min[(size_t)g * m + row] : 0.0f;
    }
  }
  __syncthreads();
  int cur = 0;
  bool full = false;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    cl.sync();   // every CTA is done reading the shared norms of the previous sweep
    // exact squared norms of the own columns, shared with every CTA
    for (int j = warp; j < 2 * bs; j += nw) {
      const int slot = j / bs, i = j % bs;
      const float* a = col(cur, slot, i);
      float s2 = 0.f;
      for (int e = 0; e < ne; ++e) s2 = fmaf(a[lane + 32 * e], a[lane + 32 * e], s2);
      s2 = warp_sum(s2);
      if (lane == 0) {
        *nrm(cur, slot, i) = s2;
        const int g = cl_block(c, slot, 0) * bs + i;
        for (int k = 0; k < kClP; ++k) cl.map_shared_rank(allnrm, k)[g] = s2;
      }
    }
    if (tid == 0) {
      s_rot = 0;
      s_rel2 = 0u;
    }
    cl.sync();
    // top set: the D columns of largest norm (ties by lower index)
    for (int g = warp; g < ng; g += nw) {
      const float ng_ = allnrm[g];
      int rk = 0;
      for (int i = lane; i < ng; i += 32) rk += (allnrm[i] > ng_) || (allnrm[i] == ng_ && i < g);
      rk = __reduce_add_sync(0xffffffffu, rk);
      if (lane == 0) top[g] = rk < D ? 1 : 0;
    }
    __syncthreads();
    bool wrot = false;   // this warp rotated in the sweep; the largest rel2 it rotated (lane 0)
    float wrel2 = 0.f;
    for (int t = 0; t < kClL; ++t) {
      const int bx = cl_block(c, 0, t), by = cl_block(c, 1, t);
      const int nrounds = t == 0 ? 2 * bs - 1 : bs;
      for (int e = tid; e < nrounds * bs; e += kClThreads) {
        const int round = e / bs, k = e % bs;
        int sp = 0, ip = k, sq = 1, iq = k + round;
        if (t == 0) {   // local indices 0 .. 2 bs - 1: slot 0 first, then slot 1
          cl_pair(2 * bs, round, k, ip, iq);
          sp = ip >= bs;
          ip -= sp ? bs : 0;
          sq = iq >= bs;
          iq -= sq ? bs : 0;
        } else {
          iq -= iq >= bs ? bs : 0;
        }
        const int gp = (sp ? by : bx) * bs + ip, gq = (sq ? by : bx) * bs + iq;
        const bool act = full || top[gp] || top[gq];
        s_pairs[round * kClBsMax + k] = act ? (sp * kClBsMax + ip) | ((sq * kClBsMax + iq) << 8) : -1;
      }
      __syncthreads();
      float* const cbase = colbuf + (size_t)cur * 2 * kClBsMax * kClStride;
      float* const nbase = bnrm + cur * 2 * kClBsMax;
      for (int round = 0; round < nrounds; ++round) {
        if (warp < bs) {
          const int e = s_pairs[round * kClBsMax + warp];
          if (e >= 0) {
            const int jp = e & 0xff, jq = e >> 8;
            float* np = nbase + jp;
            float* nq = nbase + jq;
            if (*np > 1e-30f && *nq > 1e-30f) {
              float* ap = cbase + jp * kClStride;
              float* aq = cbase + jq * kClStride;
              float rel2 = 0.f;
              const bool rot = two ? cl_rotate<true>(ap, aq, np, nq, lane, tol2, rel2)
                                   : cl_rotate<false>(ap, aq, np, nq, lane, tol2, rel2);
              if (rot) {
                wrot = true;
                wrel2 = fmaxf(wrel2, rel2);
              }
            }
          }
        }
        __syncthreads();
      }
      // pull the blocks of the next step from their holders
      cl.sync();
      const int tn = (t + 1) % kClL;
      for (int slot = 0; slot < 2; ++slot) {
        int hc, hs;
        cl_holder(cl_block(c, slot, tn), t, hc, hs);
        const float4* src = reinterpret_cast<const float4*>(cl.map_shared_rank(col(cur, hs, 0), hc));
        float4* dst = reinterpret_cast<float4*>(col(cur ^ 1, slot, 0));
        // whole columns (the zero rows too), kClStride / 4 = 64 float4 each
        for (int o = tid; o < bs * (kClStride / 4); o += kClThreads) dst[o] = src[o];
        const float* sn = cl.map_shared_rank(nrm(cur, hs, 0), hc);
        for (int i = tid; i < bs; i += kClThreads) *nrm(cur ^ 1, slot, i) = sn[i];
      }
      // a CTA's own pull must be complete before its next rounds; no cluster barrier is needed:
      // the buffer pulled into is read by others only after the next step's barrier (which
      // this CTA reaches after its pull), and the buffer pulled from is written again only
      // after that barrier too (which every reader reaches after its pull)
      __syncthreads();
      cur ^= 1;
    }
    if (lane == 0 && wrot) {
      s_rot = 1;
      atomicMax(&s_rel2, __float_as_uint(wrel2));   // non-negative floats order as their bits
    }
    __syncthreads();
    // did any CTA rotate in this sweep?
    if (tid < kClP) {
      cl.map_shared_rank(s_flags, tid)[c] = s_rot;
      cl.map_shared_rank(s_rels, tid)[c] = s_rel2;
    }
    cl.sync();
    bool any = false;
    float rel2 = 0.f;
    for (int k = 0; k < kClP; ++k) {
      any |= s_flags[k] != 0;
      rel2 = fmaxf(rel2, __uint_as_float(s_rels[k]));
    }
    // an update's core whose sweep rotated only weakly coupled pairs is done (the refinement
    // that follows takes the rest); dense calls sweep until nothing rotates
    const bool weak = use_hdr == 1 && any && rel2 < kClStopRel * kClStopRel;
    if (!full && any && !weak && sweep + 1 >= kClTopOnlySweeps) {
      // the top set keeps changing (values straddling the cut are close): every pair from here on
      full = true;
      if (use_hdr == 1 && c == 0 && tid == 0) h->jacobi_full += 1;
    }
    if (!any || weak) {
      if (full) break;
      // the norms are those of the sweep's start (nothing rotated since, or only weakly)
      float topmin = 3.0e38f, bsum = 0.f, bmax = 0.f;
      for (int g = 0; g < ng; ++g) {
        if (top[g]) {
          topmin = fminf(topmin, allnrm[g]);
        } else {
          const float a = sqrtf(allnrm[g]);
          bsum += a;
          bmax = fmaxf(bmax, a);
        }
      }
      if (bmax * bsum < 0.98f * topmin) break;
      full = true;
      if (use_hdr == 1 && c == 0 && tid == 0) {
        h->jacobi_gersh += 1;
        h->jacobi_full += 1;
      }
    }
  }
  if (use_hdr == 1 && c == 0 && tid == 0) {
    const int done = sweep < max_sweeps ? sweep + 1 : sweep;
    h->last_sweeps = done;
    h->jacobi_sweeps += done;
  }
  // a dense call that asked for it learns that the sweeps ran out before convergence
  if (use_hdr == 2 && c == 0 && tid == 0 && sweep >= max_sweeps) set_status(h, DAMF_ERR_NOT_CONVERGED);
  // exact norms, order by decreasing norm (ties by index), write the top D as E and Theta
  cl.sync();   // every CTA is done reading the shared norms of the last sweep
  for (int j = warp; j < 2 * bs; j += nw) {
    const int slot = j / bs, i = j % bs;
    const float* a = col(cur, slot, i);
    float s2 = 0.f;
    for (int e = 0; e < ne; ++e) s2 = fmaf(a[lane + 32 * e], a[lane + 32 * e], s2);
    s2 = warp_sum(s2);
    const int g = cl_block(c, slot, 0) * bs + i;
    if (lane == 0)
      for (int k = 0; k < kClP; ++k) cl.map_shared_rank(allnrm, k)[g] = g < m ? sqrtf(s2) : -1.0f;
  }
  cl.sync();
  for (int j = warp; j < 2 * bs; j += nw) {
    const int slot = j / bs, i = j % bs;
    const int g = cl_block(c, slot, 0) * bs + i;
    if (g >= m) continue;
    const float nj = allnrm[g];
    int rk = 0;
    for (int k = lane; k < m; k += 32) rk += (allnrm[k] > nj) || (allnrm[k] == nj && k < g);
    rk = __reduce_add_sync(0xffffffffu, rk);
    if (rk < D) {
      const float inv = nj > 0.f ? 1.0f / nj : 0.0f;
      const float* a = col(cur, slot, i);
      for (int row = lane; row < m; row += 32) E[row * D + rk] = a[row] * inv;
      if (lane == 0) theta[rk] = nj;
    }
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int D>
static cudaError_t cl_launch(DevHeader* h, const float* Min, int m_host, int use_hdr, float* E, float* theta,
                             int max_sweeps, cudaStream_t s) {
  cudaFuncSetAttribute(k_jacobi_cl<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmemBytes);
  k_jacobi_cl<D><<<kClP, kClThreads, kClSmemBytes, s>>>(h, Min, m_host, use_hdr, E, theta, kClTol, max_sweeps);
  return cudaGetLastError();
}

// Top-d SVD of the current update's core (m = d + nS from the device header): E, theta.
cudaError_t launch_core_svd(Ctx* c, cudaStream_t s) {
  switch (c->d) {
    case 16: return cl_launch<16>(c->hdr, c->ws.M, 0, 1, c->ws.E, c->ws.theta, 20, s);
    case 32: return cl_launch<32>(c->hdr, c->ws.M, 0, 1, c->ws.E, c->ws.theta, 20, s);
    case 64: return cl_launch<64>(c->hdr, c->ws.M, 0, 1, c->ws.E, c->ws.theta, 20, s);
    default: return cl_launch<128>(c->hdr, c->ws.M, 0, 1, c->ws.E, c->ws.theta, 20, s);
  }
}

// Top-d SVD of a dense m x m column-major matrix (m <= kMaxM): E (m x d row-major), theta.
cudaError_t cluster_svd_dense(const float* Min, int m, int d, float* E, float* theta, DevHeader* h, int report_nc,
                              cudaStream_t s) {
  if (m > kMaxM || m < d) return cudaErrorInvalidValue;
  const int mode = report_nc ? 2 : 0;
  switch (d) {
    case 16: return cl_launch<16>(h, Min, m, mode, E, theta, 30, s);
    case 32: return cl_launch<32>(h, Min, m, mode, E, theta, 30, s);
    case 64: return cl_launch<64>(h, Min, m, mode, E, theta, 30, s);
    default: return cl_launch<128>(h, Min, m, mode, E, theta, 30, s);
  }
}

}  // namespace damf
