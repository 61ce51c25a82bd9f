// Step 2 of the update on its own (Sec. 4.5 "Rediagonalization", Eq. "svd_small_edge"):
// the top-d SVD of the (d + r) x (d + r) core  M = [[diag(sigma), 0], [0, 0]] + L R^T,
// with L = [W_B; R_B] and R = [W_C; R_C] given by the caller.  The same kernels as the
// update path: one assembly kernel into a column-major scratch copy of M, the block Jacobi
// SVD on an 8-CTA cluster (jacobi_cluster.cu) and H = M^T E Theta^{-1}; then a check of the
// results (non-finite values: DAMF_ERR_NUMERIC) and, when the caller asks for it, a copy of
// the device status word into the caller's int32.
#include "damf_internal.cuh"

namespace damf {

// M[i][j] (column-major, ld m) = sigma_i [i == j < d] + sum_a L[i][a] R[j][a]
__global__ void k_assemble_lr(const float* __restrict__ sigma, const float* __restrict__ L,
                              const float* __restrict__ R, int d, int r, float* M) {
  const int m = d + r;
  const int j = blockIdx.x;
  if (j >= m) return;
  __shared__ float Rj[kMaxR];
  for (int a = threadIdx.x; a < r; a += blockDim.x) Rj[a] = R[(size_t)j * r + a];
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    float s = (i == j && i < d) ? sigma[i] : 0.0f;
    for (int a = 0; a < r; ++a) s = fmaf(L[(size_t)i * r + a], Rj[a], s);
    M[(size_t)j * m + i] = s;
  }
}

// Non-finite singular values or vectors set DAMF_ERR_NUMERIC (the first error is kept); the
// status word is then copied to `status` (device int32) when given.
__global__ void k_core_check(DevHeader* h, const float* __restrict__ E, const float* __restrict__ H,
                             const float* __restrict__ theta, int m, int d, int32_t* status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < m * d; i += blockDim.x)
    if (!isfinite(E[i]) || !isfinite(H[i])) bad = 1;
  for (int k = threadIdx.x; k < d; k += blockDim.x)
    if (!isfinite(theta[k])) bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bad) set_status(h, DAMF_ERR_NUMERIC);
    __threadfence();
    if (status) *status = *(volatile int*)&h->status;
  }
}

cudaError_t core_svd_into(const float* sigma, const float* L, const float* R, int d, int r, float* E, float* H,
                          float* theta, DevHeader* h, float* M, int32_t* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(h, 0, sizeof(DevHeader), s);
  if (e != cudaSuccess) return e;
  k_assemble_lr<<<d + r, 256, 0, s>>>(sigma, L, R, d, r, M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = jacobi_svd_dense(M, d + r, d, E, H, theta, 1, h, s)) != cudaSuccess) return e;
  k_core_check<<<1, 256, 0, s>>>(h, E, H, theta, d + r, d, status);
  return cudaGetLastError();
}

}  // namespace damf

using namespace damf;

namespace {
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
bool core_args_ok(int d, int r) { return (d == 16 || d == 32 || d == 64 || d == 128) && r >= 1 && r <= kMaxR; }
}  // namespace

extern "C" {

size_t damf_core_svd_workspace_size(int32_t d, int32_t r) {
  if (!core_args_ok(d, r)) return 0;
  return align256(sizeof(DevHeader)) + align256((size_t)(d + r) * (d + r) * sizeof(float));
}

damf_status damf_core_svd(const float* sigma, const float* L, const float* R, int32_t d, int32_t r, float* E,
                          float* H, float* theta, void* workspace, size_t workspace_bytes, int32_t* status,
                          void* stream) {
  if (!core_args_ok(d, r) || !sigma || !L || !R || !E || !H || !theta || !workspace) return DAMF_ERR_INVALID;
  if (workspace_bytes < damf_core_svd_workspace_size(d, r)) return DAMF_ERR_CAPACITY;
  DevHeader* h = (DevHeader*)workspace;
  float* M = (float*)((char*)workspace + align256(sizeof(DevHeader)));
  cudaError_t e = core_svd_into(sigma, L, R, d, r, E, H, theta, h, M, status, (cudaStream_t)stream);
  return e == cudaSuccess ? DAMF_OK : DAMF_ERR_CUDA;
}

}  // extern "C"
