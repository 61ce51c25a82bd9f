// Rediagonalisation (Step 2 of Sec. 4.5; Eq. "svd_small_edge"): the top-d SVD of the
// (d + r) x (d + r) core M by one-sided (Hestenes) Jacobi on a single CTA.
//
// The working matrix A = M J (J accumulated plane rotations, not stored) lives in
// shared memory, column-major with the column count padded to a multiple of 32 so a
// warp holds a column in m/32 registers per lane.  Each sweep visits every column pair
// once in round-robin order (m/2 disjoint pairs per round, one warp per pair); a pair
// is rotated when |a_p . a_q| > tol |a_p| |a_q|, which makes the two columns
// orthogonal.  At convergence the columns are U Theta; the top-d by norm give E and
// Theta, and the right vectors follow as H = M^T E Theta^{-1} (update.cu, k_hmat).
#include "damf_internal.cuh"

namespace damf {

constexpr int kMaxEP = kMaxM / 32;  // column elements per lane (7)

__device__ __forceinline__ void round_robin_pair(int mp, int round, int k, int& p, int& q) {
  const int L = mp - 1;
  if (k == 0) {
    p = L;
    q = round;
  } else {
    p = (round + k) % L;
    q = (round - k + L) % L;
  }
}

template <int D>
__global__ void __launch_bounds__(1024, 1) k_jacobi(DevHeader* h, const float* __restrict__ Min, int m_host, int use_hdr,
                                                    float* E, float* theta, float tol, int max_sweeps) {
  extern __shared__ float A[];
  __shared__ float nrm[kMaxM];
  __shared__ int rot_flag;
  if (h->status != 0) return;
  const int m = use_hdr ? D + h->nS : m_host;
  if (use_hdr && h->nS == 0) return;
  const int mp = (m + 31) & ~31;
  const int ep = mp / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int o = tid; o < mp * mp; o += blockDim.x) {
    const int j = o / mp, i = o % mp;
    A[o] = (i < m && j < m) ? Min[(size_t)j * m + i] : 0.0f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rot_flag = 0;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      for (int k = warp; k < mp / 2; k += nw) {
        int p, q;
        round_robin_pair(mp, round, k, p, q);
        float* ap = A + p * mp;
        float* aq = A + q * mp;
        float x[kMaxEP], y[kMaxEP];
        float aa = 0.f, bb = 0.f, gg = 0.f;
#pragma unroll
        for (int e = 0; e < kMaxEP; ++e) {
          if (e < ep) {
            x[e] = ap[lane + 32 * e];
            y[e] = aq[lane + 32 * e];
            aa = fmaf(x[e], x[e], aa);
            bb = fmaf(y[e], y[e], bb);
            gg = fmaf(x[e], y[e], gg);
          }
        }
        aa = warp_sum(aa);
        bb = warp_sum(bb);
        gg = warp_sum(gg);
        if (aa > 1e-30f && bb > 1e-30f && fabsf(gg) > tol * sqrtf(aa) * sqrtf(bb)) {
          const float zeta = (bb - aa) / (2.0f * gg);
          const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + hypotf(1.0f, zeta));
          const float c = rsqrtf(1.0f + t * t);
          const float s = c * t;
#pragma unroll
          for (int e = 0; e < kMaxEP; ++e) {
            if (e < ep) {
              ap[lane + 32 * e] = c * x[e] - s * y[e];
              aq[lane + 32 * e] = s * x[e] + c * y[e];
            }
          }
          if (lane == 0) rot_flag = 1;
        }
      }
      __syncthreads();
    }
    if (rot_flag == 0) break;
    __syncthreads();
  }
  // column norms, then order by decreasing norm (ties by index)
  for (int j = warp; j < mp; j += nw) {
    float s = 0.f;
    for (int e = 0; e < ep; ++e) {
      const float v = A[j * mp + lane + 32 * e];
      s = fmaf(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) nrm[j] = (j < m) ? sqrtf(s) : -1.0f;
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
  k_jacobi<D><<<1, 1024, sm, s>>>(c->hdr, c->ws.M, 0, 1, c->ws.E, c->ws.theta, 2e-6f, 30);
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
  k_jacobi<D><<<1, 1024, sm, s>>>(h, Min, m, 0, E, theta, 2e-6f, 40);
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
