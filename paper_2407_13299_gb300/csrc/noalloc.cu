// ozaki_gemm_noalloc: the Ozaki product of ozaki_gemm for callers that cannot
// hand the library a workspace. Its scratch (exponents, digit planes, the
// transposed B, the error flag and the tensor-core executor's partial sums)
// lives in one fixed device array defined in this file, so the call allocates
// nothing. The array exists once per GPU that loads this part of the library
// and stays until the process exits.

#include <cuda_runtime.h>

#include <mutex>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr size_t kNoAllocBytes = size_t(128) << 20;  // 128 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device. The name is only a host
// stand-in for the device symbol, so its address is looked up once per device
// (with that device current) and cached.
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DMP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DMP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DMP_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return DMP_OK;
}

}  // namespace
}  // namespace dmp

extern "C" {

int ozaki_gemm_noalloc(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int32_t mode, int32_t slices, int32_t executor,
                       void* stream) {
  size_t need = 0;
  const int rc = ozaki_gemm_workspace_size(m, n, k, mode, slices, executor, &need);
  if (rc != DMP_OK) return rc;
  if (need > dmp::kNoAllocBytes) return DMP_ERR_WORKSPACE;  // problem too large for the fixed array
  void* scratch = nullptr;
  if (need > 0) {
    const int r = dmp::noalloc_scratch(&scratch);
    if (r != DMP_OK) return r;
  }
  // Every piece of the scratch that is read is written first by this call
  // (ozaki_gemm clears its error flag itself), so nothing left by an earlier
  // call can leak into the result.
  return ozaki_gemm(m, n, k, A, lda, B, ldb, C, ldc, mode, slices, executor, scratch, dmp::kNoAllocBytes,
                    stream);
}

}  // extern "C"
