// Power-of-two row scaling and digit split (Sec. "Ozaki Scheme").
//
// For row r of A: e_r = ilogb(max_j |A_rj|) + 1 (0 for a zero row), so the
// scaled entries x = A_rj 2^-e_r lie in (-1, 1). The s digits of x are the
// beta-bit truncated base-2^beta expansion of |x| with the sign of x:
//   d_i = sign(x) * (floor(|x| 2^(beta i)) mod 2^beta),   |d_i| <= 2^beta - 1.
// They are read straight off the FP64 significand: with A_rj = m 2^(E-1075)
// (m the 53-bit significand, E the biased exponent), U = floor(|x| 2^96) is m
// shifted by E - 1075 - e_r + 96, and digit i is the beta-bit field of U that
// starts beta i bits below its top (beta s <= 72 < 96). No floating-point
// rounding is involved, so the digits are exact.
//
// Nearest digits (E4M3 mode, beta 5; BF16 mode, beta 8): the row exponent is
// one larger, so |x| < 1/2, and d_i = floor(y + 1/2) for y = 2^beta x,
// x <- y - d_i. With V = floor(x 2^95) in two's complement, the first i digits
// together are N_i = floor(V 2^-(95 - beta i) + 1/2) (the remainder after them
// lies in [-1/2, 1/2) units of their last place), so d_i = N_i - 2^beta N_(i-1)
// is a signed beta-bit field of V plus the bit below it. Bits of x below 2^-95
// never reach a rounding bit (at most 72 + 1 bits are read), so the floor is
// harmless. |d_i| <= 2^(beta-1): integers exact in E4M3 (beta 5) and in
// bfloat16 (beta 8).
//
// One CTA per row. Each thread loads pairs of adjacent entries (16-byte loads,
// 512 contiguous bytes per warp) and keeps up to 8192 entries of the row in
// registers, so the row is read from memory once: a max-reduction, then the
// digits of the same registers go to every plane (4-byte stores of two bf16 or
// 2-byte stores of two int8 digits per plane; nearest digits: four entries per
// thread). Longer rows take further sweeps that read the rest of the row again.

#include <cuda_bf16.h>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int kSplitThreads = 512;
constexpr int kPairs = 8;                                           // entry pairs a thread holds
constexpr int kSweep = 2 * kPairs * kSplitThreads;  // 8192 entries
constexpr int64_t kMaxRow = (int64_t{1} << 31) - 1 - kSweep;     // in-row offsets stay below 2^31

// U = floor(|a| 2^(96 - e_row)) as w0 (bits 64..95), w1 (32..63), w2 (0..31).
// |a| < 2^e_row for every finite entry, so U < 2^96; a row holding NaN/Inf has
// e_row = 0 and its digits are never used (the epilogue writes NaN). With
// m = mh 2^32 + ml the significand, U = m 2^t, t = E - 1075 - e_row + 96: word
// i of U is the funnel shift by t mod 32 of words i - floor(t/32) - 1 and
// i - floor(t/32) of m. Only 32-bit integer operations are used (64-bit integer
// arithmetic is slow on this GPU).
__device__ __forceinline__ void fix96(double a, int c_row, uint32_t& w0, uint32_t& w1, uint32_t& w2, bool& neg) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(a));
  const uint32_t lo = static_cast<uint32_t>(__double2loint(a));
  neg = (hi >> 31) != 0;
  const int E = static_cast<int>((hi >> 20) & 0x7ffu);
  const uint32_t mh = (hi & 0xfffffu) | (E != 0 ? 0x100000u : 0u);
  const int t = (E == 0 ? 1 : E) - c_row;  // c_row = 1075 + e_row - 96
  const int z = -(t >> 5);                 // word i of U reads words i + z - 1, i + z of m
  const uint32_t bs = static_cast<uint32_t>(t) & 31u;
  // word z + d of m for d = -1 .. 2 (m has words 0 = lo and 1 = mh)
  const uint32_t m_m1 = (z == 1) ? lo : ((z == 2) ? mh : 0u);
  const uint32_t m_0 = (z == 0) ? lo : ((z == 1) ? mh : 0u);
  const uint32_t m_1 = (z == -1) ? lo : ((z == 0) ? mh : 0u);
  const uint32_t m_2 = (z == -2) ? lo : ((z == -1) ? mh : 0u);
  w2 = __funnelshift_l(m_m1, m_0, bs);
  w1 = __funnelshift_l(m_0, m_1, bs);
  w0 = __funnelshift_l(m_1, m_2, bs);
}

// Bits [P, P + BETA) of U (P a compile-time bit position).
template <int P, int BETA>
__device__ __forceinline__ uint32_t field(uint32_t w0, uint32_t w1, uint32_t w2) {
  constexpr uint32_t mask = (1u << BETA) - 1u;
  if constexpr (P >= 64) {
    return (w0 >> (P - 64)) & mask;
  } else if constexpr (P >= 32) {
    return __funnelshift_r(w1, w0, P - 32) & mask;
  } else {
    return __funnelshift_r(w2, w1, P) & mask;
  }
}

// bfloat16 bits of sign * v for 0 <= v <= 255, in the upper half of a float:
// g = 1.5 2^23 + v is exact, and sg g - sg 1.5 2^23 is exactly +v, -v or +0
// (an exact zero sum rounds to +0), so the float holds sign * v exactly, and
// sign * v has at most 8 significant bits, so its float bits end in 16 zeros.
__device__ __forceinline__ uint32_t digit_float_bits(uint32_t v, float sg) {
  const float g = __uint_as_float(0x4B400000u | v);
  return __float_as_uint(fmaf(sg, g, -sg * 12582912.0f));
}

template <int I, int KIND, int BETA>
__device__ __forceinline__ void store_digit_pair(uint32_t a0, uint32_t a1, uint32_t a2, bool na, uint32_t b0,
                                                 uint32_t b1, uint32_t b2, bool nb, void* planes, int off) {
  constexpr int P = 96 - BETA * (I + 1);
  const uint32_t va = field<P, BETA>(a0, a1, a2);
  const uint32_t vb = field<P, BETA>(b0, b1, b2);
  if constexpr (KIND == 1) {
    const uint32_t da = na ? (0u - va) : va, db = nb ? (0u - vb) : vb;
    static_cast<uint16_t*>(planes)[off] = static_cast<uint16_t>((da & 0xffu) | ((db & 0xffu) << 8));
  } else {
    const uint32_t fa = digit_float_bits(va, na ? -1.0f : 1.0f);
    const uint32_t fb = digit_float_bits(vb, nb ? -1.0f : 1.0f);
    static_cast<uint32_t*>(planes)[off] = __byte_perm(fa, fb, 0x7632);  // high halves: (fb.hi << 16) | fa.hi
  }
}

// V = floor(a 2^(95 - e_row)) = floor(x 2^95) as a 96-bit two's complement
// integer (words v0: bits 64..95, v1, v2). The significand m of
// a = +-m 2^(E - 1075), negated in two's complement for a < 0 and sign-extended,
// is shifted by t = E - 1075 + 95 - e_row like U in fix96: left, or right,
// where dropping bits of a two's complement number is exactly the floor.
// |x| < 1/2 keeps |V| < 2^94; 32-bit operations only.
__device__ __forceinline__ void fix95_signed(double a, int c_row95, uint32_t& v0, uint32_t& v1, uint32_t& v2) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(a));
  const uint32_t lo = static_cast<uint32_t>(__double2loint(a));
  const bool neg = (hi >> 31) != 0;
  const int E = static_cast<int>((hi >> 20) & 0x7ffu);
  const uint32_t mh = (hi & 0xfffffu) | (E != 0 ? 0x100000u : 0u);
  const uint32_t s0 = neg ? (0u - lo) : lo;                          // word 0 of +-m
  const uint32_t s1 = neg ? (~mh + (lo == 0u ? 1u : 0u)) : mh;      // word 1
  const uint32_t sx = neg ? 0xffffffffu : 0u;                       // words 2, 3, ...
  const int t = (E == 0 ? 1 : E) - c_row95;  // c_row95 = 1075 + e_row - 95
  const int z = -(t >> 5);
  const uint32_t bs = static_cast<uint32_t>(t) & 31u;
  // word z + d of the sign-extended significand for d = -1 .. 2 (zero below word 0)
  auto word = [&](int d) { const int i = z + d; return i < 0 ? 0u : (i == 0 ? s0 : (i == 1 ? s1 : sx)); };
  const uint32_t m_m1 = word(-1), m_0 = word(0), m_1 = word(1), m_2 = word(2);
  v2 = __funnelshift_l(m_m1, m_0, bs);
  v1 = __funnelshift_l(m_0, m_1, bs);
  v0 = __funnelshift_l(m_1, m_2, bs);
}

// Bits [Q, Q + W) of V read as a signed W-bit number (compile-time position and width).
template <int Q, int W>
__device__ __forceinline__ int sfield(uint32_t v0, uint32_t v1, uint32_t v2) {
  uint32_t w;
  int pos;
  if constexpr (Q >= 64) {
    w = v0;
    pos = Q - 64;
  } else if constexpr (Q >= 32 && Q + W <= 64) {
    w = v1;
    pos = Q - 32;
  } else if constexpr (Q >= 32) {
    w = __funnelshift_r(v1, v0, Q - 32);
    pos = 0;
  } else if constexpr (Q + W <= 32) {
    w = v2;
    pos = Q;
  } else {
    w = __funnelshift_r(v2, v1, Q);
    pos = 0;
  }
  int r;
  asm("bfe.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(pos), "r"(W));
  return r;
}

// Nearest digit I + 1 from V: N_i = floor(V / 2^p + 1/2) at p = 95 - beta i
// is the rounding of V at that position, and d_i = N_i - 2^beta N_(i-1) works
// out to the beta-bit field [p, p + beta) of V read as a signed number plus the
// bit p - 1, i.e. (u + 1) >> 1 for the signed (beta + 1)-bit field
// u = [p - 1, p + beta). The value goes to a float exactly (1.5 2^23 + d +
// 2^(beta-1) holds d + 2^(beta-1) in its low bits). E4M3 digits (beta 5,
// |d| <= 16): a pair of floats becomes two E4M3 bytes in one conversion.
// bfloat16 digits (beta 8, |d| <= 128, at most 8 significant bits): the upper
// half of each float. Four consecutive entries (two register pairs) go to one
// 4-byte (E4M3) or 8-byte (bfloat16) store per plane: a warp writes 128 or
// 256 contiguous bytes per plane.
template <int I, int KIND, int BETA>
__device__ __forceinline__ void store_nearest4(int s, const uint32_t (&w)[4][3], char* base, int quad_off,
                                               int64_t plane_bytes) {
  if constexpr (I < kMaxSlices) {
    if (I < s) {
      constexpr int Q = 94 - BETA * (I + 1);
      constexpr uint32_t kHalf = 1u << (BETA - 1);
      float f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t dh = static_cast<uint32_t>((sfield<Q, BETA + 1>(w[u][0], w[u][1], w[u][2]) + 1 +
                                                   (1 << BETA)) >> 1);  // d + 2^(beta-1)
        f[u] = __uint_as_float(0x4B400000u | dh) - (12582912.0f + static_cast<float>(kHalf));
      }
      if constexpr (KIND == 4) {
        uint16_t lo, hi;  // upper byte from the first operand
        asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(f[1]), "f"(f[0]));
        asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(f[3]), "f"(f[2]));
        reinterpret_cast<uint32_t*>(base + I * plane_bytes)[quad_off] =
            static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
      } else {
        uint2 pk;
        pk.x = __byte_perm(__float_as_uint(f[0]), __float_as_uint(f[1]), 0x7632);
        pk.y = __byte_perm(__float_as_uint(f[2]), __float_as_uint(f[3]), 0x7632);
        reinterpret_cast<uint2*>(base + I * plane_bytes)[quad_off] = pk;
      }
      store_nearest4<I + 1, KIND, BETA>(s, w, base, quad_off, plane_bytes);
    }
  }
}

// First entry of register pair q of a thread in the sweep starting at c0:
// adjacent pairs across the threads (bf16 and int8 digits), or two adjacent
// pairs per thread (E4M3 digits, so that each thread owns four consecutive
// entries and stores 4-byte words).
template <bool QUAD, int THREADS = kSplitThreads>
__device__ __forceinline__ int entry_of(int c0, int tid, int q) {
  if constexpr (QUAD) {
    return c0 + 4 * (tid + THREADS * (q >> 1)) + 2 * (q & 1);
  } else {
    return c0 + 2 * (tid + THREADS * q);
  }
}

template <int I, int KIND, int BETA>
__device__ __forceinline__ void store_digits(int s, uint32_t a0, uint32_t a1, uint32_t a2, bool na, uint32_t b0,
                                             uint32_t b1, uint32_t b2, bool nb, char* base, int pair_off,
                                             int64_t plane_bytes) {
  if constexpr (I < kMaxSlices) {
    if (I < s) {
      store_digit_pair<I, KIND, BETA>(a0, a1, a2, na, b0, b1, b2, nb, base + I * plane_bytes, pair_off);
      store_digits<I + 1, KIND, BETA>(s, a0, a1, a2, na, b0, b1, b2, nb, base, pair_off, plane_bytes);
    }
  }
}

// frexp exponent of the row maximum from the maxima of the high words (sign
// cleared) and of the low words of its entries (0 for a zero row): a normal
// value 1.f 2^(E-1023) is 0.1f 2^(E-1022); a subnormal frac 2^-1074 with frac of
// b bits lies in [2^(b-1075), 2^(b-1074)). The largest entry has the largest
// high word; if every high word is zero, the largest low word is the largest
// subnormal.
__device__ __forceinline__ int row_exponent(uint32_t mxh, uint32_t mxl) {
  if (mxh != 0) {
    const int E = static_cast<int>(mxh >> 20);
    if (E != 0) return E - 1022;
    return (64 - __clz(static_cast<int>(mxh))) - 1074;
  }
  if (mxl != 0) return (32 - __clz(static_cast<int>(mxl))) - 1074;
  return 0;
}

// Entries j, j + 1 of the row (zero past k or for a padding row).
__device__ __forceinline__ double2 load_pair(const double* __restrict__ row, int j, int k, bool live, bool vec) {
  if (live && vec && j + 1 < k) return *reinterpret_cast<const double2*>(row + j);
  double2 v;
  v.x = (live && j < k) ? row[j] : 0.0;
  v.y = (live && j + 1 < k) ? row[j + 1] : 0.0;
  return v;
}

__device__ __forceinline__ void max_bits(double a, uint32_t& mxh, uint32_t& mxl, bool& bad) {
  const uint32_t h = static_cast<uint32_t>(__double2hiint(a)) & 0x7fffffffu;
  bad |= h >= 0x7ff00000u;
  mxh = max(mxh, h);
  mxl = max(mxl, static_cast<uint32_t>(__double2loint(a)));
}

// One row r of A (m x k, leading dimension lda) into exps[r] and the s planes
// (row length k_pad, plane_stride elements apart); one whole CTA per row.
// Offsets within a row are 32-bit (k_pad < 2^31, checked by the launcher).
// KIND 1: int8 digits, 3: bfloat16 holding the same integers, 4: E4M3 bytes.
// BETA 7: truncated digits; BETA 5 and 8: nearest digits (four entries per thread).
// S > 0: the slice count is the compile-time constant S (s is ignored), so the
// per-digit slice test folds away. THREADS threads share the row (kPairs entry
// pairs each per sweep of 2 kPairs THREADS entries).
template <int KIND, int BETA, int S = 0, int THREADS = kSplitThreads>
__device__ __forceinline__ void split_one_row(const double* __restrict__ A, int64_t r, int64_t m, int k,
                                              int64_t lda, int s_arg, int32_t* __restrict__ exps,
                                              void* __restrict__ planes, int k_pad, int64_t plane_stride,
                                              int* flag) {
  constexpr bool kNearest = BETA != 7;
  constexpr int kSweep = 2 * kPairs * THREADS;
  const int s = S > 0 ? S : s_arg;
  const int tid = threadIdx.x;
  __shared__ uint32_t red_h[THREADS / 32], red_l[THREADS / 32];
  __shared__ int red_bad[THREADS / 32];
  const bool live = r < m;
  const double* row = A + (live ? r * lda : 0);
  const bool vec = (reinterpret_cast<uintptr_t>(row) & 15) == 0;

  double2 v[kPairs];
#pragma unroll
  for (int q = 0; q < kPairs; ++q) v[q] = load_pair(row, entry_of<kNearest, THREADS>(0, tid, q), k, live, vec);
  uint32_t mxh = 0, mxl = 0;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < kPairs; ++q) {
    max_bits(v[q].x, mxh, mxl, bad);
    max_bits(v[q].y, mxh, mxl, bad);
  }
  if (live) {
    for (int j = kSweep + tid; j < k; j += THREADS) max_bits(row[j], mxh, mxl, bad);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mxh = max(mxh, __shfl_xor_sync(0xffffffffu, mxh, o));
    mxl = max(mxl, __shfl_xor_sync(0xffffffffu, mxl, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((tid & 31) == 0) {
    red_h[tid >> 5] = mxh;
    red_l[tid >> 5] = mxl;
    red_bad[tid >> 5] = bad ? 1 : 0;
  }
  __syncthreads();
  int any_bad = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    mxh = max(mxh, red_h[w]);
    mxl = max(mxl, red_l[w]);
    any_bad |= red_bad[w];
  }
  int e_row = any_bad ? 0 : row_exponent(mxh, mxl);
  if (kNearest && (mxh | mxl) != 0) ++e_row;  // nearest digits: |x| < 1/2 (a zero row keeps 0)
  if (tid == 0) {
    // a row holding NaN/Inf is marked; the product epilogue then writes NaN
    exps[r] = any_bad ? kBadExp : e_row;
    if (any_bad && flag != nullptr) atomicExch(flag, 1);
  }
  const int c_row = 1075 + e_row - 96;

  constexpr int kElemBytes = (KIND == 1 || KIND == 4) ? 1 : 2;
  char* base = static_cast<char*>(planes) + r * k_pad * kElemBytes;
  const int64_t plane_bytes = plane_stride * kElemBytes;
  for (int c0 = 0;;) {
#pragma unroll
    for (int q = 0; q < kPairs; q += (kNearest ? 2 : 1)) {
      const int j = entry_of<kNearest, THREADS>(c0, tid, q);
      if (j < k_pad) {
        if constexpr (kNearest) {
          // entries j .. j + 3 (k_pad is a multiple of 4, so all four are inside)
          uint32_t w[4][3];
          fix95_signed(v[q].x, c_row + 1, w[0][0], w[0][1], w[0][2]);
          fix95_signed(v[q].y, c_row + 1, w[1][0], w[1][1], w[1][2]);
          fix95_signed(v[q + 1].x, c_row + 1, w[2][0], w[2][1], w[2][2]);
          fix95_signed(v[q + 1].y, c_row + 1, w[3][0], w[3][1], w[3][2]);
          store_nearest4<0, KIND, BETA>(s, w, base, j >> 2, plane_bytes);
        } else {
          uint32_t a0, a1, a2, b0, b1, b2;
          bool na, nb;
          fix96(v[q].x, c_row, a0, a1, a2, na);
          fix96(v[q].y, c_row, b0, b1, b2, nb);
          store_digits<0, KIND, BETA>(s, a0, a1, a2, na, b0, b1, b2, nb, base, j >> 1, plane_bytes);
        }
      }
    }
    if (k_pad - c0 <= kSweep) break;
    c0 += kSweep;
#pragma unroll
    for (int q = 0; q < kPairs; ++q) v[q] = load_pair(row, entry_of<kNearest, THREADS>(c0, tid, q), k, live, vec);
  }
}

template <int KIND, int BETA, int S = 0>
__global__ void __launch_bounds__(kSplitThreads, 2)
split_rows_kernel(const double* __restrict__ A, int64_t m, int64_t k, int64_t lda, int s,
                  int32_t* __restrict__ exps, void* __restrict__ planes, int64_t k_pad,
                  int64_t plane_stride, int* flag, const int* done) {
  if (done != nullptr && *done) return;
  split_one_row<KIND, BETA, S>(A, blockIdx.x, m, static_cast<int>(k), lda, s, exps, planes,
                               static_cast<int>(k_pad), plane_stride, flag);
}

// The split with a compile-time slice count for the counts the purification
// uses most (INT8 digits in bf16, BF16 nearest digits, E4M3 digits), else the
// runtime count.
template <int KIND, int BETA, int S>
void launch_split_s(dim3 grid, cudaStream_t st, const double* A, int64_t m, int64_t k, int64_t lda, int s,
                    int32_t* exps, void* planes, int64_t k_pad, int64_t plane_stride, int* flag, const int* done) {
  split_rows_kernel<KIND, BETA, S><<<grid, kSplitThreads, 0, st>>>(A, m, k, lda, s, exps, planes, k_pad,
                                                                   plane_stride, flag, done);
}
template <int KIND, int BETA, int S_LO, int S_HI>
void launch_split_any(dim3 grid, cudaStream_t st, const double* A, int64_t m, int64_t k, int64_t lda, int s,
                      int32_t* exps, void* planes, int64_t k_pad, int64_t plane_stride, int* flag, const int* done) {
  if constexpr (S_LO <= S_HI) {
    if (s == S_LO) {
      launch_split_s<KIND, BETA, S_LO>(grid, st, A, m, k, lda, s, exps, planes, k_pad, plane_stride, flag, done);
      return;
    }
    launch_split_any<KIND, BETA, S_LO + 1, S_HI>(grid, st, A, m, k, lda, s, exps, planes, k_pad, plane_stride, flag,
                                                 done);
  } else {
    launch_split_s<KIND, BETA, 0>(grid, st, A, m, k, lda, s, exps, planes, k_pad, plane_stride, flag, done);
  }
}

// Grouped: CTA x covers row x - row_start[b] of matrix b (row_start ascending,
// row_start[nmats] = total padded rows). Finished matrices are skipped.
// Batch rows are short (at most about 1500 entries): 64 threads per row, so
// that many rows are in flight per SM (sixteen CTAs). Every matrix of a batch has the
// same slice count, a template argument where the launcher has an instance
// for it (S = 0: taken from the descriptor).
constexpr int kGroupedSplitThreads = 64;

template <int KIND, int BETA, int S>
__global__ void __launch_bounds__(kGroupedSplitThreads, 16)
split_grouped_kernel(const BatchMat* __restrict__ mats, const int64_t* __restrict__ row_start, int nmats,
                     int which) {
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
  split_one_row<KIND, BETA, S, kGroupedSplitThreads>(A, r, M.n, static_cast<int>(M.n), lda, M.s, exps, planes,
                                                     static_cast<int>(M.k_pad), M.n_pad * M.k_pad, nullptr);
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
  if (k > k_pad || k_pad > kMaxRow) return cudaErrorInvalidValue;
  const int64_t plane_stride = m_pad * k_pad;
  dim3 grid(static_cast<unsigned>(m_pad));
  ProfScope prof(DMP_PROF_SPLIT, st);
  if (elem_kind == 1 && beta == 7) {
    split_rows_kernel<1, 7><<<grid, kSplitThreads, 0, st>>>(A, m, k, lda, s, exps, planes, k_pad, plane_stride,
                                                            flag, done);
  } else if (elem_kind == 3 && beta == 7) {
    launch_split_any<3, 7, 4, 9>(grid, st, A, m, k, lda, s, exps, planes, k_pad, plane_stride, flag, done);
  } else if (elem_kind == 3 && beta == 8) {
    launch_split_any<3, 8, 3, 7>(grid, st, A, m, k, lda, s, exps, planes, k_pad, plane_stride, flag, done);
  } else if (elem_kind == 4 && beta == 5) {
    launch_split_any<4, 5, 5, 11>(grid, st, A, m, k, lda, s, exps, planes, k_pad, plane_stride, flag, done);
  } else {
    return cudaErrorInvalidValue;
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

template <int KIND, int BETA, int S_LO, int S_HI>
void launch_grouped_any(unsigned grid, cudaStream_t st, const BatchMat* mats, const int64_t* row_start, int nmats,
                        int which, int s) {
  if constexpr (S_LO <= S_HI) {
    if (s == S_LO) {
      split_grouped_kernel<KIND, BETA, S_LO><<<grid, kGroupedSplitThreads, 0, st>>>(mats, row_start, nmats, which);
      return;
    }
    launch_grouped_any<KIND, BETA, S_LO + 1, S_HI>(grid, st, mats, row_start, nmats, which, s);
  } else {
    split_grouped_kernel<KIND, BETA, 0><<<grid, kGroupedSplitThreads, 0, st>>>(mats, row_start, nmats, which);
  }
}

cudaError_t launch_split_grouped(const BatchMat* mats, const int64_t* row_start, int nmats, int64_t total_rows,
                                 int which, int beta, int s, cudaStream_t st) {
  if (total_rows <= 0) return cudaSuccess;
  ProfScope prof(DMP_PROF_SPLIT, st);  // batch rows are at most a few thousand long (k_pad << kMaxRow)
  const unsigned grid = static_cast<unsigned>(total_rows);
  if (beta == 7) {
    launch_grouped_any<3, 7, 4, 9>(grid, st, mats, row_start, nmats, which, s);
  } else if (beta == 8) {
    launch_grouped_any<3, 8, 3, 7>(grid, st, mats, row_start, nmats, which, s);
  } else if (beta == 5) {
    launch_grouped_any<4, 5, 5, 11>(grid, st, mats, row_start, nmats, which, s);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace dmp
