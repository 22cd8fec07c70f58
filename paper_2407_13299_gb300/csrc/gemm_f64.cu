// FP64 executor: C = A B in float64 with the FP64 tensor-core MMA
// (mma.sync m8n8k4 f64). This is the plain double-precision purification the
// Ozaki modes are measured against, and the FP64 mode of ozaki_gemm.
//
// 64 x 64 output tile per CTA, 4 warps in 2 x 2, 32 x 32 per warp, K blocks of
// 16 staged through shared memory with a two-stage cp.async pipeline. A and B
// are read with bounds checks (any m, n, k, leading dimension).

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int THREADS = 128;
constexpr int APAD = 4;  // row padding (doubles) against bank conflicts
constexpr int BPAD = 4;

struct Params {
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  int64_t m, n, k;
  int sym, tiles_n, T;
  EpiArgs epi;
  const int* done;
};

__device__ __forceinline__ void mma_f64(double* c, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(THREADS) gemm_f64_kernel(const Params p) {
  if (p.done != nullptr && *p.done) return;
  __shared__ double As[2][BM][BK + APAD];
  __shared__ double Bs[2][BK][BN + BPAD];

  int bi, bj;
  if (p.sym) {
    upper_tile(blockIdx.x, p.T, bi, bj);
  } else {
    bi = blockIdx.x / p.tiles_n;
    bj = blockIdx.x % p.tiles_n;
  }
  const int64_t m0 = static_cast<int64_t>(bi) * BM;
  const int64_t n0 = static_cast<int64_t>(bj) * BN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, tig = lane & 3;

  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

  const int KT = static_cast<int>((p.k + BK - 1) / BK);
  double ra[8], rb[8];
  auto gload = [&](int kt) {
    const int64_t k0 = static_cast<int64_t>(kt) * BK;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * THREADS;  // 0..1023
      {
        const int row = e / BK, col = e % BK;
        const int64_t gr = m0 + row, gc = k0 + col;
        ra[q] = (gr < p.m && gc < p.k) ? p.A[gr * p.lda + gc] : 0.0;
      }
      {
        const int row = e / BN, col = e % BN;
        const int64_t gr = k0 + row, gc = n0 + col;
        rb[q] = (gr < p.k && gc < p.n) ? p.B[gr * p.ldb + gc] : 0.0;
      }
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * THREADS;
      As[buf][e / BK][e % BK] = ra[q];
      Bs[buf][e / BN][e % BN] = rb[q];
    }
  };

  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < KT; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < KT) gload(kt + 1);
#pragma unroll
    for (int kk = 0; kk < BK / 4; ++kk) {
      double af[4], bf[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) af[mi] = As[buf][wm * 32 + mi * 8 + g][kk * 4 + tig];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) bf[ni] = Bs[buf][kk * 4 + tig][wn * 32 + ni * 8 + g];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_f64(acc[mi][ni], af[mi], bf[ni]);
    }
    if (kt + 1 < KT) sstore(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int64_t r = m0 + wm * 32 + mi * 8 + g;
        const int64_t c = n0 + wn * 32 + ni * 8 + 2 * tig + q;
        // symmetric output: written once from r <= c and mirrored
        if (p.sym && r > c) continue;
        if (r < p.m && c < p.n) epi_apply(p.epi, r, c, acc[mi][ni][q], p.sym && r < c);
      }
}

}  // namespace

cudaError_t launch_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m,
                            int64_t n, int64_t k, int sym, const EpiArgs& epi, const int* done,
                            cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  Params p;
  p.A = A;
  p.lda = lda;
  p.B = B;
  p.ldb = ldb;
  p.m = m;
  p.n = n;
  p.k = k;
  p.sym = sym;
  p.tiles_n = static_cast<int>((n + BN - 1) / BN);
  p.T = static_cast<int>((m + BM - 1) / BM);
  p.epi = epi;
  p.done = done;
  const int tiles_m = static_cast<int>((m + BM - 1) / BM);
  const int ntiles = sym ? p.T * (p.T + 1) / 2 : tiles_m * p.tiles_n;
  ProfScope prof(DMP_PROF_PRODUCT, st);
  gemm_f64_kernel<<<ntiles, THREADS, 0, st>>>(p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dmp
