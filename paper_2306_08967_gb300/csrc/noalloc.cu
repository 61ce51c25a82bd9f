// damf_core_svd_noalloc: the core SVD of damf_core_svd for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc or hand us a workspace: for example an engine
// plugin that receives only its input and output pointers from a host framework whose
// allocator owns all device memory, or code on a latency-critical path where cudaMalloc
// (which may synchronise the device) is not allowed.  This entry point keeps its scratch
// (a status word and the assembled core M) in one file-scope device array of fixed size,
// so it allocates nothing.  Limits and sharing rules are stated in include/damf.h.
#include "damf_internal.cuh"

namespace damf {
cudaError_t core_svd_into(const float* sigma, const float* L, const float* R, int d, int r, float* E, float* H,
                          float* theta, DevHeader* h, float* M, int32_t* status, cudaStream_t s);
}  // namespace damf

using namespace damf;

namespace {

constexpr size_t kHeaderBytes = 1024;
static_assert(sizeof(DevHeader) <= kHeaderBytes, "status area too small");
// status word area + the largest core (d + r <= 256) in FP32: 263,168 bytes
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)kMaxM * kMaxM * sizeof(float);

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_core_scratch[kScratchBytes];

}  // namespace

extern "C" damf_status damf_core_svd_noalloc(const float* sigma, const float* L, const float* R, int32_t d,
                                             int32_t r, float* E, float* H, float* theta, int32_t* status,
                                             void* stream) {
  if (!(d == 16 || d == 32 || d == 64 || d == 128) || !sigma || !L || !R || !E || !H || !theta)
    return DAMF_ERR_INVALID;
  if (r < 1 || r > kMaxR) return DAMF_ERR_CAPACITY;   // the scratch holds cores up to (128 + 128)^2
  // The host-side name of the array is not a device address: look the address up, with the
  // caller's device current.  The first lookup on a device loads the library's device code
  // there (set-up; make that first call before any stream capture); later lookups only read
  // it back, and looking it up on every call keeps the address right after a device reset
  // (which unloads the code and may place the array elsewhere when it is loaded again).
  void* base = nullptr;
  if (cudaGetSymbolAddress(&base, g_core_scratch) != cudaSuccess || base == nullptr) return DAMF_ERR_CUDA;
  DevHeader* h = (DevHeader*)base;
  float* M = (float*)((char*)base + kHeaderBytes);
  // core_svd_into clears the status word before use; M is fully overwritten by the assembly
  const cudaError_t e = core_svd_into(sigma, L, R, d, r, E, H, theta, h, M, status, (cudaStream_t)stream);
  return e == cudaSuccess ? DAMF_OK : DAMF_ERR_CUDA;
}
