// Rediagonalisation (Step 2 of Sec. 4.5; Eq. "svd_small_edge"): entry points of the core
// SVD. The top-d SVD itself runs on an 8-CTA cluster (jacobi_cluster.cu); the right vectors
// follow from the left ones as H = M^T E Theta^{-1} (k_hmat in update.cu for the update's
// core, k_hmat_dense here for a dense matrix).
#include "damf_internal.cuh"

namespace damf {

cudaError_t launch_core_svd(Ctx* c, cudaStream_t s);
cudaError_t cluster_svd_dense(const float* Min, int m, int d, float* E, float* theta, DevHeader* h, int report_nc,
                              cudaStream_t s);
cudaError_t launch_assemble(Ctx* c, cudaStream_t s);

// M of the current update, then its top-d SVD (m = d + nS from the device header).
cudaError_t launch_core(Ctx* c, cudaStream_t s) {
  cudaError_t e = launch_assemble(c, s);
  if (e != cudaSuccess) return e;
  return launch_core_svd(c, s);
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
                              int report_nc, cudaStream_t s) {
  cudaError_t e = cluster_svd_dense(Min, m, D, E, theta, h, report_nc, s);
  if (e != cudaSuccess) return e;
  k_hmat_dense<D><<<m, 128, 0, s>>>(h, Min, m, E, theta, H);
  return cudaGetLastError();
}

cudaError_t jacobi_svd_dense(const float* Min, int m, int d, float* E, float* H, float* theta, int report_nc,
                             DevHeader* h, cudaStream_t s) {
  if (m > kMaxM || m < d) return cudaErrorInvalidValue;
  switch (d) {
    case 16: return dense_impl<16>(Min, m, E, H, theta, h, report_nc, s);
    case 32: return dense_impl<32>(Min, m, E, H, theta, h, report_nc, s);
    case 64: return dense_impl<64>(Min, m, E, H, theta, h, report_nc, s);
    default: return dense_impl<128>(Min, m, E, H, theta, h, report_nc, s);
  }
}

}  // namespace damf
