// Step 2 of the update on its own (Sec. 4.5 "Rediagonalization", Eq. "svd_small_edge"):
// the top-d SVD of the (d + r) x (d + r) core  M = [[diag(sigma), 0], [0, 0]] + L R^T,
// with L = [W_B; R_B] and R = [W_C; R_C] given by the caller.  The same kernels as the
// update path: one assembly kernel into a column-major scratch copy of M, the one-CTA
// Jacobi SVD (jacobi.cu) and H = M^T E Theta^{-1}.
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

cudaError_t core_svd_into(const float* sigma, const float* L, const float* R, int d, int r, float* E, float* H,
                          float* theta, DevHeader* h, float* M, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(h, 0, sizeof(DevHeader), s);
  if (e != cudaSuccess) return e;
  k_assemble_lr<<<d + r, 256, 0, s>>>(sigma, L, R, d, r, M);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return jacobi_svd_dense(M, d + r, d, E, H, theta, nullptr, h, s);
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
                          float* H, float* theta, void* workspace, size_t workspace_bytes, void* stream) {
  if (!core_args_ok(d, r) || !sigma || !L || !R || !E || !H || !theta || !workspace) return DAMF_ERR_INVALID;
  if (workspace_bytes < damf_core_svd_workspace_size(d, r)) return DAMF_ERR_CAPACITY;
  DevHeader* h = (DevHeader*)workspace;
  float* M = (float*)((char*)workspace + align256(sizeof(DevHeader)));
  cudaError_t e = core_svd_into(sigma, L, R, d, r, E, H, theta, h, M, (cudaStream_t)stream);
  return e == cudaSuccess ? DAMF_OK : DAMF_ERR_CUDA;
}

}  // extern "C"
