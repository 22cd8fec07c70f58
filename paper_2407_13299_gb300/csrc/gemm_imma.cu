// IMMA executor for the Ozaki slice-pair products (Sec. "Ozaki Scheme", Fig. 2).
//
// One CTA computes a 128 x 128 output tile. For each level L = s+1 down to 2 it
// forms S_L = sum_{i+j=L} D_i^A (D_j^B)^T exactly with int8 x int8 -> int32
// mma.sync (m16n8k32). Up to four consecutive levels are combined exactly in
// int64 registers, T = sum S_L 2^(7 (L_a - L)) < 2^53; at the end of each group
// its exact value T 2^(-7 L_a) is added to a float64 sum kept in shared memory,
// groups from the smallest to the largest -- the operation sequence of the
// definition, so the float64 result is reproducible bit for bit. The tile is
// then unscaled by 2^(e_r + f_c) and handed to the epilogue.
//
// Operands are zero-padded digit planes [s][rows_pad][k_pad] (K contiguous).
// The K loop runs over (level, pair, 64-wide K block) and is fed by a 4-stage
// cp.async pipeline into XOR-swizzled shared memory (conflict-free ldmatrix).
// 8 warps in a 2 x 4 grid, 64 x 32 outputs per warp.

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;  // BK in int8 elements (= bytes)
constexpr int STAGES = 4;
constexpr int THREADS = 256;
constexpr int TILE_BYTES = BM * BK;  // 8 KiB per operand tile
constexpr int PIPE_BYTES = STAGES * 2 * TILE_BYTES;
constexpr int SMEM_BYTES = PIPE_BYTES + 64 * THREADS * 8;  // + float64 group sums, [element][thread]

__device__ __forceinline__ uint32_t swz(int row, int chunk) {
  return static_cast<uint32_t>(row * 64 + ((chunk ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                            uint32_t saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(saddr));
}

__device__ __forceinline__ void mma_s8(int32_t* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Pos {
  int L, i, kt;
};

__device__ __forceinline__ void pos_first(Pos& p, int s) {
  p.L = s + 1;
  p.i = 1;
  p.kt = 0;
}
// Advance over (level, pair, K block): K blocks fastest, then pairs i of the
// level (j = L - i), then levels from s+1 down to 2.
__device__ __forceinline__ void pos_next(Pos& p, int s, int KT) {
  if (++p.kt < KT) return;
  p.kt = 0;
  const int i_hi = min(s, p.L - 1);
  if (++p.i <= i_hi) return;
  --p.L;
  p.i = max(1, p.L - s);
}

struct Params {
  const int8_t* A;
  const int8_t* B;
  int64_t psa, psb;  // plane strides (elements)
  int64_t k_pad;
  const int32_t* ea;
  const int32_t* eb;
  int64_t m, n;
  int s, beta, sym, tiles_n, T;
  EpiArgs epi;
  const int* done;
};

__global__ void __launch_bounds__(THREADS, 1) ozaki_imma_kernel(const Params p) {
  if (p.done != nullptr && *p.done) return;
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(smem));

  int bi, bj;
  if (p.sym) {
    upper_tile(blockIdx.x, p.T, bi, bj);
  } else {
    bi = blockIdx.x / p.tiles_n;
    bj = blockIdx.x % p.tiles_n;
  }
  const int64_t m0 = static_cast<int64_t>(bi) * BM;
  const int64_t n0 = static_cast<int64_t>(bj) * BN;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int wm = warp >> 2;  // 0..1
  const int wn = warp & 3;   // 0..3
  const int s = p.s;
  const int KT = static_cast<int>(p.k_pad / BK);
  const int total = KT * (s * (s + 1) / 2);

  int32_t acc[4][4][4];
  long long accT[4][4][4];  // exact sum of the current group of levels
  double* dsum = reinterpret_cast<double*>(smem + PIPE_BYTES);  // element e at dsum[e * THREADS + tid]
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[a][b][q] = 0;
        accT[a][b][q] = 0;
      }

  auto load_stage = [&](int stage, const Pos& ps) {
    const int8_t* gA = p.A + static_cast<int64_t>(ps.i - 1) * p.psa + m0 * p.k_pad + static_cast<int64_t>(ps.kt) * BK;
    const int8_t* gB = p.B + static_cast<int64_t>(ps.L - ps.i - 1) * p.psb + n0 * p.k_pad + static_cast<int64_t>(ps.kt) * BK;
    const uint32_t sA = sbase + stage * 2 * TILE_BYTES;
    const uint32_t sB = sA + TILE_BYTES;
#pragma unroll
    for (int c = tid; c < BM * 4; c += THREADS) {
      const int row = c >> 2, ch = c & 3;
      cp_async16(sA + swz(row, ch), gA + row * p.k_pad + ch * 16);
      cp_async16(sB + swz(row, ch), gB + row * p.k_pad + ch * 16);
    }
  };

  Pos lp, cp;
  pos_first(lp, s);
  pos_first(cp, s);
#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) {
    if (st < total) {
      load_stage(st, lp);
      pos_next(lp, s, KT);
    }
    cp_async_commit();
  }

  const int q8 = lane >> 3;
  for (int t = 0; t < total; ++t) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    {
      const int tn = t + STAGES - 1;
      if (tn < total) {
        load_stage(tn % STAGES, lp);
        pos_next(lp, s, KT);
      }
      cp_async_commit();
    }
    const uint32_t sA = sbase + (t % STAGES) * 2 * TILE_BYTES;
    const uint32_t sB = sA + TILE_BYTES;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[4][4];
      uint32_t bf[4][2];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int row = wm * 64 + mi * 16 + (q8 & 1) * 8 + (lane & 7);
        ldmatrix_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], sA + swz(row, 2 * ks + (q8 >> 1)));
      }
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        const int row = wn * 32 + nj * 16 + (q8 >> 1) * 8 + (lane & 7);
        ldmatrix_x4(bf[2 * nj][0], bf[2 * nj][1], bf[2 * nj + 1][0], bf[2 * nj + 1][1],
                    sB + swz(row, 2 * ks + (q8 & 1)));
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_s8(acc[mi][ni], af[mi], bf[ni]);
    }
    // end of a level: fold the exact level sum into the group sum
    if (cp.kt == KT - 1 && cp.i == min(s, cp.L - 1)) {
      const int gpos = (s + 1 - cp.L) & 3;
      const bool gend = (gpos == 3) && (cp.L != 2);
      const bool first_group = (s + 1 - cp.L) < 4;
      const double gscale = ldexp(1.0, -7 * (cp.L + gpos));
      const int g = lane >> 2, tig = lane & 3;
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (p.epi.kind == EPI_LEVELS) {
              const int64_t r = m0 + wm * 64 + mi * 16 + g + ((q >> 1) << 3);
              const int64_t c = n0 + wn * 32 + ni * 8 + 2 * tig + (q & 1);
              if (r < p.m && c < p.n)
                p.epi.levels[static_cast<int64_t>(cp.L - 2) * p.m * p.n + r * p.n + c] = acc[mi][ni][q];
            } else {
              const long long T = (gpos > 0 ? accT[mi][ni][q] : 0ll) +
                                  (static_cast<long long>(acc[mi][ni][q]) << (7 * gpos));
              if (gend) {
                const int e = (mi * 4 + ni) * 4 + q;
                const double gv = static_cast<double>(T) * gscale;
                dsum[e * THREADS + tid] = first_group ? gv : dsum[e * THREADS + tid] + gv;
              }
              accT[mi][ni][q] = T;
            }
            acc[mi][ni][q] = 0;
          }
    }
    pos_next(cp, s, KT);
  }
  cp_async_wait<0>();

  if (p.epi.kind == EPI_LEVELS) return;
  const int g = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t r = m0 + wm * 64 + mi * 16 + g + ((q >> 1) << 3);
        const int64_t c = n0 + wn * 32 + ni * 8 + 2 * tig + (q & 1);
        // symmetric output: each pair (r, c), (c, r) is written once from r <= c,
        // so the result is exactly symmetric even where A B is not (P X2)
        if (p.sym && r > c) continue;
        const bool mirror = p.sym && r < c;
        if (r < p.m && c < p.n) {
          // finish the last group (levels 2 .. L_a) and add the earlier groups
          const int La = 2 + ((s - 1) & 3);
          const double gv = static_cast<double>(accT[mi][ni][q]) * ldexp(1.0, -7 * La);
          const int e = (mi * 4 + ni) * 4 + q;
          const double acc64 = (s <= 4) ? gv : dsum[e * THREADS + tid] + gv;
          const int32_t er = p.ea[r], ec = p.eb[c];
          const double v = (er == kBadExp || ec == kBadExp) ? __longlong_as_double(0x7ff8000000000000ll)
                                                            : ldexp(acc64, er + ec);
          epi_apply(p.epi, r, c, v, mirror);
        }
      }
}

}  // namespace

cudaError_t launch_ozaki_imma(const int8_t* A, const int8_t* B, const int32_t* ea, const int32_t* eb,
                              int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                              int s, int beta, int sym, const EpiArgs& epi, const int* done,
                              cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  // set before every launch: the attribute belongs to the kernel as loaded in
  // the current context (a context created anew starts from the default)
  cudaError_t e = cudaFuncSetAttribute(ozaki_imma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  Params p;
  p.A = A;
  p.B = B;
  p.psa = m_pad * k_pad;
  p.psb = n_pad * k_pad;
  p.k_pad = k_pad;
  p.ea = ea;
  p.eb = eb;
  p.m = m;
  p.n = n;
  p.s = s;
  p.beta = beta;
  p.sym = sym;
  p.tiles_n = static_cast<int>(n_pad / BN);
  p.T = static_cast<int>(m_pad / BM);
  p.epi = epi;
  p.done = done;
  const int tiles_m = static_cast<int>(m_pad / BM);
  const int ntiles = sym ? p.T * (p.T + 1) / 2 : tiles_m * p.tiles_n;
  ProfScope prof(DMP_PROF_PRODUCT, st);
  ozaki_imma_kernel<<<ntiles, THREADS, SMEM_BYTES, st>>>(p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dmp
