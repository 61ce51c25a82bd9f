// Rediagonalisation (Step 2 of Sec. 4.5; Eq. "svd_small_edge"): the top-d SVD of the
// (d + r) x (d + r) core M by one-sided (Hestenes) Jacobi on a single CTA.
//
// The working matrix A = M J (J accumulated plane rotations, not stored) lives in
// shared memory, column-major with the column count padded to a multiple of 32 so a
// warp holds a column in m/32 registers per lane.  Each sweep visits every column pair
// once in round-robin order (m/2 disjoint pairs per round, one warp per pair); a pair
// is rotated when |a_p . a_q| > tol |a_p| |a_q|, which makes the two columns
// orthogonal.  A warp works on 4 pairs at once (8 lanes per pair, float4 accesses), which
// shares the reduction and the rotation arithmetic of a pair across 4 pairs; the kernel
// is bound by instruction issue.  Squared column norms are cached in shared memory and updated by each
// rotation (|a_p'|^2 = |a_p|^2 - t g, |a_q'|^2 = |a_q|^2 + t g), so a pair costs one
// warp reduction; they are recomputed exactly at the start of every sweep.
// Only pairs with at least one column among the current top-d (by norm) are rotated:
// when the top columns are mutually orthogonal and orthogonal to all others,
// A^T A is block diagonal, so M^T M J_top = J_top Theta_top^2 and the top columns are
// exactly the top-d singular vectors (given theta_d > every other column norm).  The
// discarded block's internal structure, which holds the slowest-converging clustered
// singular values, is never resolved; this cuts the sweep count roughly in half.  The
// premise is checked at convergence (Gershgorin bound on the discarded block's Gram
// against the smallest top norm^2); when the gap is too small to certify it the kernel
// continues with sweeps over every pair.  At convergence the columns are U Theta; the top-d by norm give E and
// Theta, and the right vectors follow as H = M^T E Theta^{-1} (update.cu, k_hmat).
#include "damf_internal.cuh"

namespace damf {

constexpr int kMaxC = kMaxM / 32;   // float4 chunks per lane of an 8-lane group (7)
constexpr int kJacobiThreads = 768;   // 96 pairs in flight: one pass per round for d + r <= 192
// A pair is rotated while |a_p . a_q| > tol |a_p| |a_q|; FP32 dot products of length <= 224
// carry relative noise of a few 1e-7, so the tolerance sits a little above that floor.
constexpr float kJacobiTol = 1e-6f;
// sweeps restricted to pairs touching the top-d set before falling back to every pair
constexpr int kTopOnlySweeps = 6;

// Circle-method pairing: in round t (0 <= t < mp-1) pair k is (mp-1, t) for k = 0 and
// ((t+k) mod (mp-1), (t-k) mod (mp-1)) otherwise; every column appears once per round.
// Both arguments of the modulo lie in [0, 2(mp-1)), so one conditional subtraction does.
__device__ __forceinline__ void round_robin_pair(int mp, int round, int k, int& p, int& q) {
  const int L = mp - 1;
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

template <int D>
__global__ void __launch_bounds__(kJacobiThreads, 2) k_jacobi(DevHeader* h, const float* __restrict__ Min, int m_host, int use_hdr,
                                                    float* E, float* theta, float tol, int max_sweeps) {
  extern __shared__ float A[];
  __shared__ float nrm[kMaxM];   // squared column norms, refreshed every sweep
  __shared__ unsigned char top[kMaxM];
  __shared__ int rot_flag;
  if (h->status != 0) return;
  const int m = use_hdr ? D + h->nS : m_host;
  if (use_hdr && h->nS == 0) return;
  const int mp = (m + 31) & ~31;
  const int ep = mp / 32;
  const int nc = mp / 32;   // float4 chunks per lane of an 8-lane group, per column
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int grp = lane >> 3, gl = lane & 7;
  for (int o = tid; o < mp * mp; o += blockDim.x) {
    const int j = o / mp, i = o % mp;
    A[o] = (i < m && j < m) ? Min[(size_t)j * m + i] : 0.0f;
  }
  __syncthreads();
  const float tol2 = tol * tol;
  __shared__ int full_mode;    // 0: only pairs touching the top-d set; 1: every pair
  __shared__ float gersh, topmin, bsum, bmax;
  if (tid == 0) full_mode = 0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = warp; j < mp; j += nw) {
      float s2 = 0.f;
      for (int e = 0; e < ep; ++e) {
        const float v = A[j * mp + lane + 32 * e];
        s2 = fmaf(v, v, s2);
      }
      s2 = warp_sum(s2);
      if (lane == 0) nrm[j] = s2;
    }
    if (tid == 0) rot_flag = 0;
    __syncthreads();
    // the D columns of largest norm are the current "top" set
    for (int j = warp; j < mp; j += nw) {
      const float nj = nrm[j];
      int rk = 0;
      for (int i = lane; i < mp; i += 32) {
        const float ni = nrm[i];
        rk += (ni > nj) || (ni == nj && i < j);
      }
      for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
      if (lane == 0) top[j] = rk < D ? 1 : 0;
    }
    __syncthreads();
    const bool full = full_mode != 0;
    for (int round = 0; round < mp - 1; ++round) {
      // 4 pairs per warp, 8 lanes per pair; lane gl of a group holds rows 4 (gl + 8 c) .. +3
      for (int kb = warp * 4; kb < mp / 2; kb += nw * 4) {
        const int k = kb + grp;
        int p = 0, q = 0;
        if (k < mp / 2) round_robin_pair(mp, round, k, p, q);
        const float aa = nrm[p], bb = nrm[q];
        const bool act = k < mp / 2 && (full || (top[p] | top[q])) && aa > 1e-30f && bb > 1e-30f;
        float4* ap = reinterpret_cast<float4*>(A + p * mp);
        float4* aq = reinterpret_cast<float4*>(A + q * mp);
        // pass 1: dot product (columns are read again for the rotation, keeping the
        // register footprint small enough for 768 threads beside a push)
        float2 g01 = make_float2(0.f, 0.f), g23 = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < kMaxC; ++c) {
          if (c < nc && act) {
            const float4 x = ap[gl + 8 * c];
            const float4 y = aq[gl + 8 * c];
            g01 = __ffma2_rn(make_float2(x.x, x.y), make_float2(y.x, y.y), g01);
            g23 = __ffma2_rn(make_float2(x.z, x.w), make_float2(y.z, y.w), g23);
          }
        }
        float gg = (g01.x + g01.y) + (g23.x + g23.y);
        gg += __shfl_xor_sync(0xffffffffu, gg, 1);
        gg += __shfl_xor_sync(0xffffffffu, gg, 2);
        gg += __shfl_xor_sync(0xffffffffu, gg, 4);
        if (act && gg * gg > tol2 * aa * bb) {
          // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / (2 g): the smaller
          // root of t^2 + 2 zeta t - 1 = 0, so the rotated columns are orthogonal
          const float zeta = __fdividef(bb - aa, 2.0f * gg);
          const float az = fabsf(zeta);
          const float ta = az < 1e15f ? __frcp_rn(az + __fsqrt_rn(fmaf(az, az, 1.0f))) : __fdividef(0.5f, az);
          const float t = copysignf(ta, zeta);
          const float cs = rsqrtf(fmaf(t, t, 1.0f));
          const float sn = cs * t;
          const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ms2 = make_float2(-sn, -sn);
          // pass 2: rotate
#pragma unroll
          for (int c = 0; c < kMaxC; ++c) {
            if (c < nc) {
              const float4 x = ap[gl + 8 * c];
              const float4 y = aq[gl + 8 * c];
              const float2 xl = make_float2(x.x, x.y), xh = make_float2(x.z, x.w);
              const float2 yl = make_float2(y.x, y.y), yh = make_float2(y.z, y.w);
              const float2 pl = __ffma2_rn(c2, xl, __fmul2_rn(ms2, yl));
              const float2 ph = __ffma2_rn(c2, xh, __fmul2_rn(ms2, yh));
              const float2 ql = __ffma2_rn(s2, xl, __fmul2_rn(c2, yl));
              const float2 qh = __ffma2_rn(s2, xh, __fmul2_rn(c2, yh));
              ap[gl + 8 * c] = make_float4(pl.x, pl.y, ph.x, ph.y);
              aq[gl + 8 * c] = make_float4(ql.x, ql.y, qh.x, qh.y);
            }
          }
          if (gl == 0) {
            nrm[p] = fmaxf(aa - t * gg, 0.0f);
            nrm[q] = bb + t * gg;
            rot_flag = 1;
          }
        }
      }
      __syncthreads();
    }
    if (!full && sweep + 1 >= kTopOnlySweeps && rot_flag != 0) {
      // the top set keeps changing (singular values straddling the cut are too close):
      // resolve every pair from here on
      if (tid == 0) {
        full_mode = 1;
        if (use_hdr) h->jacobi_full += 1;
      }
    }
    if (rot_flag == 0) {
      if (full) break;
      // top-only convergence is exact when every eigenvalue of the discarded block's
      // Gram is below the smallest top norm^2; Gershgorin row sums bound those
      // eigenvalues.  Otherwise fall back to rotating every pair.
      if (tid == 0) {
        gersh = 0.f;
        topmin = 3.0e38f;
        bsum = 0.f;
        bmax = 0.f;
      }
      __syncthreads();
      // cheap bound first: row sums of |G_bot| <= max_j |a_j| * sum_i |a_i| (Cauchy-Schwarz)
      for (int j = tid; j < m; j += blockDim.x) {
        if (top[j]) {
          atomicMin((int*)&topmin, __float_as_int(nrm[j]));
        } else {
          const float nj = sqrtf(nrm[j]);
          atomicAdd(&bsum, nj);
          atomicMax((int*)&bmax, __float_as_int(nj));
        }
      }
      __syncthreads();
      if (bmax * bsum < 0.98f * topmin) break;
      if (tid == 0 && use_hdr) h->jacobi_gersh += 1;
      // exact Gershgorin row sums of the discarded block's Gram
      for (int j = warp; j < m; j += nw) {
        if (top[j]) continue;
        float row = 0.f;
        for (int i = 0; i < m; ++i) {
          if (top[i]) continue;
          float dv = 0.f;
          for (int e = 0; e < ep; ++e) dv = fmaf(A[j * mp + lane + 32 * e], A[i * mp + lane + 32 * e], dv);
          row += fabsf(warp_sum(dv));
        }
        if (lane == 0) atomicMax((int*)&gersh, __float_as_int(row));
      }
      __syncthreads();
      if (gersh < 0.98f * topmin) break;
      if (tid == 0) {
        full_mode = 1;
        if (use_hdr) h->jacobi_full += 1;
      }
    }
    __syncthreads();
  }
  if (tid == 0 && use_hdr) {
    h->last_sweeps = sweep + 1;
    h->jacobi_sweeps += sweep + 1;
  }
  // exact column norms, then order by decreasing norm (ties by index)
  for (int j = warp; j < mp; j += nw) {
    float s2 = 0.f;
    for (int e = 0; e < ep; ++e) {
      const float v = A[j * mp + lane + 32 * e];
      s2 = fmaf(v, v, s2);
    }
    s2 = warp_sum(s2);
    if (lane == 0) nrm[j] = (j < m) ? sqrtf(s2) : -1.0f;
  }
  __syncthreads();
  for (int j = warp; j < m; j += nw) {
    const float nj = nrm[j];
    int rk = 0;
    for (int i = lane; i < m; i += 32) {
      const float ni = nrm[i];
      rk += (ni > nj) || (ni == nj && i < j);
    }
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    if (rk < D) {
      const float inv = nj > 0.f ? 1.0f / nj : 0.0f;
      for (int i = lane; i < m; i += 32) E[i * D + rk] = A[j * mp + i] * inv;
      if (lane == 0) theta[rk] = nj;
    }
  }
}

// Jacobi on the core of the current update (m = D + nS from the device header).
template <int D>
static cudaError_t core_impl(Ctx* c, cudaStream_t s) {
  const size_t sm = (size_t)kMaxM * kMaxM * sizeof(float);
  cudaFuncSetAttribute(k_jacobi<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_jacobi<D><<<1, kJacobiThreads, sm, s>>>(c->hdr, c->ws.M, 0, 1, c->ws.E, c->ws.theta, kJacobiTol, 20);
  return cudaGetLastError();
}

cudaError_t launch_assemble(Ctx* c, cudaStream_t s);

cudaError_t launch_core(Ctx* c, cudaStream_t s) {
  cudaError_t e = launch_assemble(c, s);
  if (e != cudaSuccess) return e;
  switch (c->d) {
    case 16: return core_impl<16>(c, s);
    case 32: return core_impl<32>(c, s);
    case 64: return core_impl<64>(c, s);
    default: return core_impl<128>(c, s);
  }
}

// H = M^T E Theta^{-1} for a dense m x m column-major M (initialisation path).
template <int D>
__global__ void k_hmat_dense(DevHeader* h, const float* __restrict__ M, int m, const float* __restrict__ E,
                             const float* __restrict__ theta, float* H) {
  if (h->status != 0) return;
  const int j = blockIdx.x;
  if (j >= m) return;
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < m; ++i) s = fmaf(M[(size_t)j * m + i], E[i * D + k], s);
    const float t = theta[k];
    H[j * D + k] = t > 0.f ? s / t : 0.0f;
  }
}

template <int D>
static cudaError_t dense_impl(const float* Min, int m, float* E, float* H, float* theta, DevHeader* h,
                              cudaStream_t s) {
  const size_t sm = (size_t)kMaxM * kMaxM * sizeof(float);
  cudaFuncSetAttribute(k_jacobi<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_jacobi<D><<<1, kJacobiThreads, sm, s>>>(h, Min, m, 0, E, theta, kJacobiTol, 30);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hmat_dense<D><<<m, 128, 0, s>>>(h, Min, m, E, theta, H);
  return cudaGetLastError();
}

cudaError_t jacobi_svd_dense(const float* Min, int m, int d, float* E, float* H, float* theta, float*, DevHeader* h,
                             cudaStream_t s) {
  if (m > kMaxM || m < d) return cudaErrorInvalidValue;
  switch (d) {
    case 16: return dense_impl<16>(Min, m, E, H, theta, h, s);
    case 32: return dense_impl<32>(Min, m, E, H, theta, h, s);
    case 64: return dense_impl<64>(Min, m, E, H, theta, h, s);
    default: return dense_impl<128>(Min, m, E, H, theta, h, s);
  }
}

}  // namespace damf
