// ozaki_gemm_noalloc: the Ozaki product of ozaki_gemm for callers that cannot
// hand the library a workspace. Its scratch (exponents, digit planes, the
// transposed B, the error flag and the tensor-core executor's partial sums)
// lives in one fixed device array defined in this file, so the call allocates
// nothing. The array exists once per GPU that loads this part of the library
// and stays until the process exits.

#include <cuda_runtime.h>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr size_t kNoAllocBytes = size_t(128) << 20;  // 128 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array in the current context. In host code the
// array's name is only a stand-in for the device symbol, so the address is
// looked up with cudaGetSymbolAddress -- on every call, not cached: a context
// that is torn down and created again (cudaDeviceReset, or a caller's own
// driver-API context on the same device) loads the library's device code at a
// new address, and a pointer kept from the old context would point at memory
// that no longer belongs to the array. The lookup is a host-side table query
// of the runtime; it allocates nothing and enqueues no work.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DMP_ERR_CUDA;
  *out = p;
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
