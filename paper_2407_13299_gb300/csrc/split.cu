// Power-of-two row scaling and digit split (Sec. "Ozaki Scheme").
//
// For row r of A: e_r = ilogb(max_j |A_rj|) + 1 (0 for a zero row), so the
// scaled entries x = A_rj 2^-e_r lie in (-1, 1). The s digits of x are the
// beta-bit truncated base-2^beta expansion of |x| with the sign of x:
//   d_i = sign(x) * (floor(|x| 2^(beta i)) mod 2^beta),   |d_i| <= 2^beta - 1.
// They are read straight off the FP64 significand: with A_rj = m 2^(E-1075)
// (m the 53-bit significand, E the biased exponent), floor(|x| 2^(beta s)) is
// m shifted by E - 1075 - e_r + beta s, and digit i is a beta-bit field of it.
// No floating-point rounding is involved, so the digits are exact.
//
// One CTA per row: a max-reduction pass over the row, then a pass that emits
// eight consecutive elements per thread into every plane with one vector store
// per plane (8 bytes for int8, 16 bytes for 16-bit digits). The row is read
// twice; the second read is served from L2.

#include <cuda_bf16.h>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int kSplitThreads = 256;

__device__ __forceinline__ void digits_of(double a, int e_row, int s, int beta, int32_t* d) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(a));
  const bool neg = (bits >> 63) != 0;
  const int E = static_cast<int>((bits >> 52) & 0x7ff);
  const unsigned long long frac = bits & ((1ull << 52) - 1);
  const unsigned long long mant = (E == 0) ? frac : (frac | (1ull << 52));
  const int ex = (E == 0) ? 1 : E;
  // |A_rj| 2^(beta s - e_r) = mant 2^shift, below 2^(beta s) <= 2^72
  const int shift = ex - 1075 - e_row + beta * s;
  unsigned __int128 T = 0;
  if (mant != 0) {
    if (shift >= 0) {
      T = static_cast<unsigned __int128>(mant) << shift;
    } else if (shift > -64) {
      T = static_cast<unsigned __int128>(mant >> (-shift));
    }
  }
  const unsigned long long mask = (1ull << beta) - 1;
#pragma unroll
  for (int i = 0; i < kMaxSlices; ++i) {
    if (i < s) {
      const int v = static_cast<int>(static_cast<unsigned long long>(T >> (beta * (s - 1 - i))) & mask);
      d[i] = neg ? -v : v;
    }
  }
}

// One row r of A (m x k, leading dimension lda) into exps[r] and the s planes;
// called by one whole CTA of kSplitThreads threads.
template <int KIND>  // 1: int8, 2: int16, 3: bfloat16 holding the same integers
__device__ __forceinline__ void split_one_row(const double* __restrict__ A, int64_t r, int64_t m, int64_t k,
                                              int64_t lda, int s, int beta, int32_t* __restrict__ exps,
                                              void* __restrict__ planes, int64_t k_pad, int64_t plane_stride,
                                              int* flag) {
  const int tid = threadIdx.x;
  __shared__ unsigned long long red[kSplitThreads / 32];
  __shared__ int e_sh;

  unsigned long long mx = 0;
  bool bad = false;
  if (r < m) {
    const double* row = A + r * lda;
    for (int64_t j = tid; j < k; j += kSplitThreads) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(row[j])) & 0x7fffffffffffffffull;
      bad |= (b >> 52) == 0x7ff;
      mx = b > mx ? b : mx;  // bit patterns of nonnegative doubles order like their values
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  if (bad && flag != nullptr) atomicExch(flag, 1);
  __shared__ int bad_sh;
  if (tid == 0) bad_sh = 0;
  __syncthreads();
  if (bad) atomicExch(&bad_sh, 1);
  __syncthreads();
  if (tid == 0) {
    unsigned long long v = 0;
    for (int w = 0; w < kSplitThreads / 32; ++w) v = red[w] > v ? red[w] : v;
    int e = 0;
    if (v != 0 && !bad_sh) frexp(__longlong_as_double(static_cast<long long>(v)), &e);
    e_sh = e;
    // a row holding NaN/Inf is marked; the product epilogue then writes NaN
    exps[r] = bad_sh ? kBadExp : e;
  }
  __syncthreads();
  const int e_row = e_sh;

  const double* row = A + r * lda;
  for (int64_t j0 = static_cast<int64_t>(tid) * 8; j0 < k_pad; j0 += kSplitThreads * 8) {
    uint32_t pk[kMaxSlices][4];
#pragma unroll
    for (int i = 0; i < kMaxSlices; ++i) pk[i][0] = pk[i][1] = pk[i][2] = pk[i][3] = 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t j = j0 + q;
      const double a = (r < m && j < k) ? row[j] : 0.0;
      int32_t d[kMaxSlices];
      digits_of(a, e_row, s, beta, d);
#pragma unroll
      for (int i = 0; i < kMaxSlices; ++i) {
        if (i < s) {
          if (KIND == 1) {
            pk[i][q >> 2] |= (static_cast<uint32_t>(d[i]) & 0xffu) << (8 * (q & 3));
          } else if (KIND == 2) {
            pk[i][q >> 1] |= (static_cast<uint32_t>(d[i]) & 0xffffu) << (16 * (q & 1));
          } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(d[i]));  // exact: |d| <= 255
            const uint32_t hb = static_cast<uint32_t>(__bfloat16_as_ushort(h));
            pk[i][q >> 1] |= hb << (16 * (q & 1));
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kMaxSlices; ++i) {
      if (i < s) {
        if (KIND == 1) {
          int8_t* dst = static_cast<int8_t*>(planes) + i * plane_stride + r * k_pad + j0;
          *reinterpret_cast<uint2*>(dst) = make_uint2(pk[i][0], pk[i][1]);
        } else {
          int16_t* dst = static_cast<int16_t*>(planes) + i * plane_stride + r * k_pad + j0;
          *reinterpret_cast<uint4*>(dst) = make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
        }
      }
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(kSplitThreads)
split_rows_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda, int s, int beta,
                  int32_t* __restrict__ exps, void* __restrict__ planes, int64_t k_pad,
                  int64_t plane_stride, int* flag, const int* done) {
  if (done != nullptr && *done) return;
  split_one_row<KIND>(A, blockIdx.x, m, k, lda, s, beta, exps, planes, k_pad, plane_stride, flag);
}

// Grouped: CTA x covers row x - row_start[b] of matrix b (row_start ascending,
// row_start[nmats] = total padded rows). Finished matrices are skipped.
template <int KIND>
__global__ void __launch_bounds__(kSplitThreads)
split_grouped_kernel(const BatchMat* __restrict__ mats, const int64_t* __restrict__ row_start, int nmats,
                     int which, int beta) {
  const int64_t x = blockIdx.x;
  int lo = 0, hi = nmats - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_start[mid] <= x) lo = mid; else hi = mid - 1;
  }
  const BatchMat& M = mats[lo];
  if (M.state->done) return;
  const int64_t r = x - row_start[lo];
  const double* A = which == 2 ? M.X2 : M.buf[which];
  const int64_t lda = which == 0 ? M.ldp : M.n;
  int32_t* exps = which == 2 ? M.expsX : M.expsP;
  void* planes = which == 2 ? M.planesX : M.planesP;
  split_one_row<KIND>(A, r, M.n, M.n, lda, M.s, beta, exps, planes, M.k_pad, M.n_pad * M.k_pad, nullptr);
}

__global__ void transpose_kernel(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                 double* __restrict__ At) {
  __shared__ double tile[32][33];
  const int64_t bx = static_cast<int64_t>(blockIdx.x) * 32;  // column block of A
  const int64_t by = static_cast<int64_t>(blockIdx.y) * 32;  // row block of A
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t r = by + yy, c = bx + threadIdx.x;
    if (r < m && c < n) tile[yy][threadIdx.x] = A[r * lda + c];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t r = bx + yy, c = by + threadIdx.x;  // At is n x m
    if (r < n && c < m) At[r * m + c] = tile[threadIdx.x][yy];
  }
}

}  // namespace

cudaError_t launch_split_rows(const double* A, int64_t m, int64_t k, int64_t lda, int s, int beta,
                              int32_t* exps, void* planes, int64_t m_pad, int64_t k_pad,
                              int elem_kind, int* flag, const int* done, cudaStream_t st) {
  if (m_pad <= 0 || k_pad <= 0) return cudaSuccess;
  const int64_t plane_stride = m_pad * k_pad;
  dim3 grid(static_cast<unsigned>(m_pad));
  ProfScope prof(DMP_PROF_SPLIT, st);
  if (elem_kind == 1) {
    split_rows_kernel<1><<<grid, kSplitThreads, 0, st>>>(A, m, k, lda, s, beta, exps, planes, k_pad,
                                                         plane_stride, flag, done);
  } else if (elem_kind == 2) {
    split_rows_kernel<2><<<grid, kSplitThreads, 0, st>>>(A, m, k, lda, s, beta, exps, planes, k_pad,
                                                         plane_stride, flag, done);
  } else {
    split_rows_kernel<3><<<grid, kSplitThreads, 0, st>>>(A, m, k, lda, s, beta, exps, planes, k_pad,
                                                         plane_stride, flag, done);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_transpose(const double* A, int64_t m, int64_t n, int64_t lda, double* At,
                             cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((m + 31) / 32));
  ProfScope prof(DMP_PROF_OTHER, st);
  transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(A, m, n, lda, At);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_grouped(const BatchMat* mats, const int64_t* row_start, int nmats, int64_t total_rows,
                                 int which, int beta, cudaStream_t st) {
  if (total_rows <= 0) return cudaSuccess;
  ProfScope prof(DMP_PROF_SPLIT, st);
  split_grouped_kernel<3><<<static_cast<unsigned>(total_rows), kSplitThreads, 0, st>>>(mats, row_start, nmats,
                                                                                       which, beta);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dmp
