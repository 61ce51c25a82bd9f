// Query (Sec. 4.6) and the periodic fold of the transforms into the bases.
//
// Fold: the paper merges successive projections into P (Sec. 4.1); over many updates P
// and P^{-1} drift from exact inverses and U = Ub PU from orthonormality.  Every
// `refold_every` updates the library re-bases:
//   R_U^T R_U = PU^T (Ub^T Ub) PU,  R_V likewise          (U = Ub PU R_U^{-1} orthonormal)
//   R_U Sigma R_V^T = E' Sigma' H'^T                      (small SVD, jacobi.cu)
//   T_U = PU R_U^{-1} E',  T_V = PV R_V^{-1} H'
//   Ub <- Ub T_U, Vb <- Vb T_V, Sigma <- Sigma', PU = PV = I.
// The represented product U Sigma V^T is unchanged.  The PPR state follows the signal:
// Xb = Ub diag(s0) maps by T_X = diag(1/s0) T_U diag(s0'), so Zb <- Zb T_X, r <- r T_X
// (PPR is linear in the signal), then s0 <- sqrt(Sigma') and the next push checks all rows.
#include "damf_internal.cuh"

namespace damf {

cudaError_t gemm_tall_scaled(const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                             const float* ascale, const float* cscale, cudaStream_t s);
cudaError_t chol_inv_upper2(const float* G, int K, float* R, float* Rinv, DevHeader* h, cudaStream_t s);
cudaError_t small_mm(const float* A, const float* B, float* C, int K, cudaStream_t s);

// rows-list query: out[i] = (base[rows[i]] * pre) P * post   (16 rows per CTA)
template <int D>
__global__ void __launch_bounds__(256) k_query_rows(const int32_t* __restrict__ rows, int count, int n, DevHeader* h,
                                                    const float* __restrict__ base, const float* __restrict__ P,
                                                    const float* __restrict__ pre, const float* __restrict__ post,
                                                    float* out) {
  extern __shared__ float smem[];
  float* Ps = smem;
  float* A = smem + D * D;
  const int r0 = blockIdx.x * 16;
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) Ps[i] = P[i];
  for (int o = threadIdx.x; o < 16 * D; o += blockDim.x) {
    const int rr = o / D, k = o % D;
    float v = 0.f;
    if (r0 + rr < count) {
      const int row = rows ? rows[r0 + rr] : r0 + rr;
      if (row >= 0 && row < n) {
        v = base[(size_t)row * D + k];
        if (pre) v *= pre[k];
      } else if (k == 0) {
        set_status(h, DAMF_ERR_INVALID);   // out-of-range id: zero row, status recorded
      }
    }
    A[o] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 16 * D; o += blockDim.x) {
    const int rr = o / D, j = o % D;
    if (r0 + rr >= count) continue;
    float s = 0.f;
    for (int k = 0; k < D; ++k) s = fmaf(A[rr * D + k], Ps[k * D + j], s);
    out[(size_t)(r0 + rr) * D + j] = post ? s * post[j] : s;
  }
}

__global__ void k_vec_prep(const float* sigma, const float* s0, float* sqsig, float* is0, int d) {
  const int k = threadIdx.x;
  if (k < d) {
    sqsig[k] = sqrtf(fmaxf(sigma[k], 0.0f));
    is0[k] = s0[k] > 0.f ? 1.0f / s0[k] : 0.0f;
  }
}

template <int D>
static cudaError_t query_rows_impl(const int32_t* rows, int count, int n, DevHeader* h, const float* base,
                                   const float* P, const float* pre, const float* post, float* out, cudaStream_t s) {
  const size_t sm = (size_t)(D * D + 16 * D) * sizeof(float);
  cudaFuncSetAttribute(k_query_rows<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_query_rows<D><<<(count + 15) / 16, 256, sm, s>>>(rows, count, n, h, base, P, pre, post, out);
  return cudaGetLastError();
}

static cudaError_t query_one(Ctx* c, const int32_t* rows, int count, const float* base, const float* P,
                             const float* pre, const float* post, float* out, cudaStream_t s) {
  if (!rows) return gemm_ctx(c, base, c->d, count, P, c->d, c->d, out, c->d, pre, post, s);
  switch (c->d) {
    case 16: return query_rows_impl<16>(rows, count, c->n, c->hdr, base, P, pre, post, out, s);
    case 32: return query_rows_impl<32>(rows, count, c->n, c->hdr, base, P, pre, post, out, s);
    case 64: return query_rows_impl<64>(rows, count, c->n, c->hdr, base, P, pre, post, out, s);
    default: return query_rows_impl<128>(rows, count, c->n, c->hdr, base, P, pre, post, out, s);
  }
}

cudaError_t launch_query(Ctx* c, const int32_t* rows, int count, float* X, float* Y, float* Z, float* sigma,
                         cudaStream_t s) {
  const int d = c->d;
  float* sqsig = c->ws.tmp;            // scratch vectors (tmp is 4 d x d)
  float* is0 = c->ws.tmp + d;
  k_vec_prep<<<1, 128, 0, s>>>(c->sigma, c->s0, sqsig, is0, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || count <= 0) goto tail;
  if (X && (e = query_one(c, rows, count, c->Ub, c->PU, nullptr, sqsig, X, s)) != cudaSuccess) return e;
  if (Y && (e = query_one(c, rows, count, c->Vb, c->PV, nullptr, sqsig, Y, s)) != cudaSuccess) return e;
  if (Z && (e = query_one(c, rows, count, c->Zb, c->PU, is0, sqsig, Z, s)) != cudaSuccess) return e;
tail:
  if (sigma) e = cudaMemcpyAsync(sigma, c->sigma, sizeof(float) * d, cudaMemcpyDeviceToDevice, s);
  return e;
}

// ---- fold ----
__global__ void k_congruence(const float* G, const float* P, float* out, float* tmp, int d) {
  // out = P^T G P (one CTA; tmp d x d scratch)
  for (int o = threadIdx.x; o < d * d; o += blockDim.x) {
    const int i = o / d, j = o % d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(G[i * d + k], P[k * d + j], s);
    tmp[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < d * d; o += blockDim.x) {
    const int i = o / d, j = o % d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(P[k * d + i], tmp[k * d + j], s);
    out[o] = s;
  }
}

// C = R_U diag(sigma) R_V^T written column-major (Jacobi input)
__global__ void k_fold_core(const float* RU, const float* RV, const float* sigma, float* Mcol, int d) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < d * d; o += gridDim.x * blockDim.x) {
    const int i = o / d, j = o % d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(RU[i * d + k] * sigma[k], RV[j * d + k], s);
    Mcol[j * d + i] = s;
  }
}

// T_X = diag(1/s0) T_U diag(sqrt(theta)); then s0 <- sqrt(theta), sigma <- theta, P's <- I
__global__ void k_fold_finish(const float* TU, float* TX, float* s0, float* sigma, const float* theta, float* PU,
                              float* PUi, float* PV, float* PVi, int d, DevHeader* h) {
  for (int o = threadIdx.x; o < d * d; o += blockDim.x) {
    const int i = o / d, j = o % d;
    const float a = s0[i] > 0.f ? 1.0f / s0[i] : 0.0f;
    TX[o] = a * TU[o] * sqrtf(fmaxf(theta[j], 0.f));
  }
  __syncthreads();
  for (int o = threadIdx.x; o < d * d; o += blockDim.x) {
    const float v = (o / d == o % d) ? 1.0f : 0.0f;
    PU[o] = PUi[o] = PV[o] = PVi[o] = v;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    sigma[k] = theta[k];
    s0[k] = sqrtf(fmaxf(theta[k], 0.f));
  }
  if (threadIdx.x == 0) {
    h->folds += 1;
    h->check_all = 1;   // the next push seeds every row (the base changed under all of them)
  }
}


cudaError_t launch_fold(Ctx* c, cudaStream_t s) {
  const int d = c->d;
  const size_t dd = (size_t)d * d;
  cudaError_t e;
  float* GU = c->ws.gram;
  float* GV = c->ws.gram + dd;
  // scratch: KU.. KVi and tmp (4 dd) are free between updates
  float* RU = c->ws.KU;
  float* RUi = c->ws.KV;
  float* RV = c->ws.KUi;
  float* RVi = c->ws.KVi;
  float* T1 = c->ws.tmp;
  float* T2 = c->ws.tmp + dd;
  float* TU = c->ws.tmp + 2 * dd;
  float* TV = c->ws.tmp + 3 * dd;
  if ((e = gram_tall(c, c->Ub, d, c->n, d, GU, s)) != cudaSuccess) return e;
  if ((e = gram_tall(c, c->Vb, d, c->n, d, GV, s)) != cudaSuccess) return e;
  k_congruence<<<1, 1024, 0, s>>>(GU, c->PU, T1, T2, d);
  if ((e = chol_inv_upper2(T1, d, RU, RUi, c->hdr, s)) != cudaSuccess) return e;
  k_congruence<<<1, 1024, 0, s>>>(GV, c->PV, T1, T2, d);
  if ((e = chol_inv_upper2(T1, d, RV, RVi, c->hdr, s)) != cudaSuccess) return e;
  k_fold_core<<<(int)((dd + 255) / 256), 256, 0, s>>>(RU, RV, c->sigma, c->ws.M, d);
  // E', theta, H' of the d x d core
  if ((e = jacobi_svd_dense(c->ws.M, d, d, c->ws.E, c->ws.H, c->ws.theta, 0, c->hdr, s)) != cudaSuccess) return e;
  // T_U = PU RUi E', T_V = PV RVi H'
  if ((e = small_mm(c->PU, RUi, T1, d, s)) != cudaSuccess) return e;
  if ((e = small_mm(T1, c->ws.E, TU, d, s)) != cudaSuccess) return e;
  if ((e = small_mm(c->PV, RVi, T1, d, s)) != cudaSuccess) return e;
  if ((e = small_mm(T1, c->ws.H, TV, d, s)) != cudaSuccess) return e;
  k_fold_finish<<<1, 1024, 0, s>>>(TU, T2, c->s0, c->sigma, c->ws.theta, c->PU, c->PUi, c->PV, c->PVi, d, c->hdr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // in-place re-basing of the four n x d arrays
  if ((e = gemm_ctx(c, c->Ub, d, c->n, TU, d, d, c->Ub, d, nullptr, nullptr, s)) != cudaSuccess) return e;
  if ((e = gemm_ctx(c, c->Vb, d, c->n, TV, d, d, c->Vb, d, nullptr, nullptr, s)) != cudaSuccess) return e;
  if ((e = gemm_ctx(c, c->Zb, d, c->n, T2, d, d, c->Zb, d, nullptr, nullptr, s)) != cudaSuccess) return e;
  if ((e = gemm_ctx(c, c->r, d, c->n, T2, d, d, c->r, d, nullptr, nullptr, s)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace damf
