// Optional kernel timing (dmp_profile_*): CUDA events recorded on the
// launching stream around each library launch, summed per kernel class.

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

struct Rec {
  cudaEvent_t a, b;
  int kind;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_pool;  // events are created once and reused after a reset
size_t g_used = 0;

}  // namespace

ProfScope::ProfScope(int kind, cudaStream_t st) : st_(st), idx_(-1) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;  // not in graphs
  if (g_used == g_pool.size()) {
    Rec r;
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
      cudaEventDestroy(r.a);
      return;
    }
    g_pool.push_back(r);
  }
  idx_ = static_cast<int>(g_used++);
  g_pool[idx_].kind = kind;
  cudaEventRecord(g_pool[idx_].a, st_);
}

ProfScope::~ProfScope() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_pool[idx_].b, st_);
}

}  // namespace dmp

using namespace dmp;

extern "C" {

int dmp_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return DMP_OK;
}

int dmp_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_used = 0;
  return DMP_OK;
}

int dmp_profile_read(int32_t kind, double* total_ms, long long* launches) {
  if (total_ms == nullptr || launches == nullptr) return DMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0.0;
  long long c = 0;
  for (size_t i = 0; i < g_used; ++i) {
    if (g_pool[i].kind != kind) continue;
    if (cudaEventSynchronize(g_pool[i].b) != cudaSuccess) return DMP_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_pool[i].a, g_pool[i].b) != cudaSuccess) return DMP_ERR_CUDA;
    t += ms;
    ++c;
  }
  *total_ms = t;
  *launches = c;
  return DMP_OK;
}

}  // extern "C"
