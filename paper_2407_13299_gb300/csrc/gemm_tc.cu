// tcgen05 executor for the Ozaki slice-pair products (Sec. "Ozaki Scheme", Fig. 2).
//
// The digits are small integers (|d| <= 127 for the truncated beta = 7 digits,
// <= 128 for the nearest beta = 8 digits), exactly representable in bfloat16,
// so the slice-pair products run on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, bf16 x bf16 -> fp32 in tensor memory). The nearest
// digits of the E4M3 mode (beta = 5, |d| <= 16) are exact E4M3 values and run
// on kind::f8f6f4 at twice the rate, with the same shared-memory layout in
// bytes (a 128-byte swizzle row holds 128 of them instead of 64). An fp32 sum
// of such products is exact while every partial sum stays at most 2^24 in
// magnitude; the K loop is therefore cut into chunks of 1024 (beta = 7 and 8:
// 1024 * 128^2 = 2^24) or 65536 (beta = 5: 65536 * 16^2 = 2^24, so a whole
// level is one chunk) K elements. Each chunk lands in one of two TMEM
// accumulators; while the tensor core fills the other, eight epilogue warps
// drain the finished one into exact int32 level sums in registers. Up to G
// consecutive levels (G = 4 for beta 7 and 5, 3 for beta 8) are combined
// exactly in int64 and the groups are added in float64 from L = s+1 down to 2
// -- the same operation sequence as the definition, so the float64 result is
// bit-for-bit the one the IMMA executor and the oracle produce.
//
// CTA layout (320 threads, one CTA per SM):
//   warp 0      TMA producer: A tile 128 x 64 and B tile BN x 64 bf16 per stage,
//               128-byte swizzle, into a 4- or 6-stage shared-memory ring
//   warp 1      TMEM owner and MMA issuer (one thread): 4 MMAs of K = 16 per
//               stage, commits free the stage and publish finished chunks
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one output
//               row per thread) and half of the BN columns
// Output tile 128 x BN (BN = 256; 128 or 256 in the batched path). In
// symmetric mode only tiles holding some element with row <= column run; each
// element with row <= column is accumulated and written once, and mirrored.
//
// Every mbarrier wait is bounded by a %globaltimer deadline; on expiry the CTA
// raises an error flag, drains what it has in flight (bounded again), frees
// its TMEM and returns.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;       // bf16 elements per K block: one 128-byte swizzle row
constexpr int TC_ROW_BYTES = 128;  // bytes of one K block row (the swizzle atom width)
constexpr int TC_MMA_PER_ATOM = 4;  // MMAs per K block: 32 bytes of K each (16 bf16 or 32 e4m3)
constexpr int TC_THREADS = 320;
constexpr int TC_EPI_WARPS = 8;
constexpr int kTileRing = 4;  // WALK 2: tile indices the producer may announce ahead

// PAIR: a cluster of two CTAs computes a 256 x BN tile with tcgen05.mma.cta_group::2;
// each CTA stages its own 128 rows of A and half of the BN rows of B, and its
// TMEM receives its 128 output rows with all BN columns.
// A PAIR stage holds two 64-element K atoms of each operand (8 MMAs per stage
// barrier round: with 4 the per-stage wait and commit left the tensor pipe
// idle about a third of the time).
template <int BN, bool PAIR = false, bool F8 = false>
struct TcCfg {
  static constexpr int KSUB = PAIR ? 2 : 1;  // K atoms (128-byte rows) per stage
  static constexpr int ATOM_K = F8 ? 128 : TC_BK;  // K elements per atom
  static constexpr int A_ATOM = TC_BM * TC_ROW_BYTES;
  static constexpr int B_ATOM = (PAIR ? BN / 2 : BN) * TC_ROW_BYTES;
  static constexpr int A_BYTES = KSUB * A_ATOM;
  static constexpr int B_BYTES = KSUB * B_ATOM;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = PAIR ? 3 : (BN == 128 ? 6 : 4);
  static constexpr int TMEM_COLS = 2 * BN;      // two fp32 chunk accumulators
  static constexpr int COLS = BN / 2;           // columns per epilogue thread
  static constexpr int BAR_BYTES = 256;
  static constexpr int SMEM = STAGES * STAGE_BYTES + BAR_BYTES + 1024;  // + alignment slack
};

struct TcParams {
  int s, beta, KT, CH, ntiles;
  int group;        // levels combined exactly per int64 group: 4 (beta 7, 5) or 3 (beta 8)
  double* scratch;  // per-CTA float64 partial sums, TC_BM * BN doubles per CTA
  int64_t m, n;
  int64_t rows_a, rows_b;  // padded rows per digit plane
  int sym, tiles_m, tiles_n;
  // tile order: bands of band_w column blocks, each cut into groups of group_h
  // row blocks, so the tiles in flight together form a near-square block and
  // share their operand panels in L2 (band_w = 0: column-major order)
  int band_w, group_h;
  const int32_t* ea;
  const int32_t* eb;
  EpiArgs epi;
  const int* done;
  int* err;
  unsigned long long timeout_ns;
  int stall_test;  // withhold each CTA's first stage (the bounded-wait test; see dmp_test_stall_next_product)
  // split launches (fewer tiles than CTAs or CTA pairs): every tile is cut
  // into split_unit_count units of one fp32 chunk, shared out in contiguous
  // ranges over all CTAs (CTA pairs)
  int split_unit_count;
  int* tile_counter;  // WALK 2: next tile to take (zeroed before the launch)
  long long* split_area;  // per (tile, CTA rank in the pair): two TC_BM x BN int64 group sums
  int* split_cnt;         // per (tile, rank, epilogue warp): contributors counted in
  // grouped mode (batched purification): tiles of many matrices in one launch
  const BatchMat* mats;  // nullptr: the single matrix above
  const int4* tiles;     // {matrix, bi, bj, 0}
  int phase;             // 0: X2 = P P;  1: P' = update(P, X2, P X2)
  int cur;               // the iterate is mats[.].buf[cur]
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(dst), "l"(tm), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* tm) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tm) : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// ---- the CTA pair (cluster of two, cta_group::2)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the shared::cluster address of the same object in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_cta(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, "
      "p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// arrive on a barrier of either CTA of the pair (a shared::cluster address).
// Used only to hand a TMEM buffer back to the MMA issuer: the loads from it
// have completed (tcgen05.wait::ld) and are ordered before the arrive by
// tcgen05.fence::before_thread_sync, and no memory this thread wrote is passed
// on through the barrier. The arrive therefore keeps the default CTA-scope
// release: a cluster-scope release adds a fence on every drained chunk that
// waits for the thread's outstanding memory operations.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
// TMA load into this CTA's shared memory that signals `bar`, which may be the peer's
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(tm), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_e4m3_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// one MMA of the 256-row pair tile: A rows from both CTAs, B halves from both
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on `bar` in both CTAs of the pair when the MMAs issued so far complete
__device__ __forceinline__ void umma_commit_pair_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(static_cast<unsigned short>(3))
      : "memory");
}
__device__ __forceinline__ void umma_commit_pair_self(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Scratch accesses with an L2 evict-last policy: the fold buffers are touched
// once per level while gigabytes of operand tiles stream through L2.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void st_keep(void* p, long long v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
// 64-bit load from L2 (.cg: not through this SM's L1, which may hold a line
// from before a reduction at L2)
__device__ __forceinline__ long long ld_l2(const void* p, uint64_t pol) {
  long long v;
  asm volatile("ld.global.cg.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// 64-bit integer add performed at L2 (no value returned, so no round trip):
// two's complement, so it adds signed values exactly
__device__ __forceinline__ void red_add_keep(void* p, long long v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

// RN(h 2^sh + l) 2^e2 as a double, for integers |h|, |l| < 2^53, 0 <= sh < 64
// and a normal result, by integer arithmetic alone: the exact sum is formed in
// 128 bits, its leading 53 bits are rounded to nearest-even, and the exponent
// and sign are set directly. This is the value float64 arithmetic gives for
// double(h) 2^(sh + e2) + double(l) 2^e2 (both products exact, one rounding),
// without the int64-to-double conversions and multiplies, which on this GPU
// run on the narrow FP64 pipe.
__device__ __forceinline__ double round_exact(long long h, int sh, long long l, int e2) {
  // x = h 2^sh + l in two's complement (xh:xl)
  const unsigned long long hl = static_cast<unsigned long long>(h) << sh;
  unsigned long long xh = sh == 0 ? static_cast<unsigned long long>(h >> 63)
                                  : static_cast<unsigned long long>(h >> (64 - sh));
  const unsigned long long xl = hl + static_cast<unsigned long long>(l);
  xh += static_cast<unsigned long long>(l >> 63) + (xl < hl ? 1ull : 0ull);
  const bool neg = static_cast<long long>(xh) < 0;
  // magnitude (mh:ml)
  const unsigned long long ml = neg ? ~xl + 1ull : xl;
  const unsigned long long mh = neg ? ~xh + (ml == 0 ? 1ull : 0ull) : xh;
  if ((mh | ml) == 0) return 0.0;
  int msb = mh != 0 ? 127 - __clzll(static_cast<long long>(mh)) : 63 - __clzll(static_cast<long long>(ml));
  unsigned long long mant;
  if (msb <= 52) {
    mant = ml << (52 - msb);  // exact (mh is zero)
  } else {
    const int r = msb - 52;  // 1 .. 63: the dropped bits all lie in ml
    mant = (ml >> r) | (r == 0 ? 0ull : mh << (64 - r));
    const unsigned long long rem = ml & ((1ull << r) - 1ull);
    const unsigned long long half = 1ull << (r - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++msb;
      }
    }
  }
  const unsigned long long bits = (neg ? (1ull << 63) : 0ull) |
                                  (static_cast<unsigned long long>(msb + e2 + 1023) << 52) |
                                  (mant & ((1ull << 52) - 1ull));
  return __longlong_as_double(static_cast<long long>(bits));
}

// RN(h 2^sh + l) as a double (unscaled), for integers |h|, |l| < 2^53 and
// 0 <= sh < 64: when the exact sum fits in 63 bits (|h| < 2^(62 - sh), always
// so for a last group of one level) it is formed in int64 and converted with
// one correctly rounded conversion; otherwise round_exact forms it in 128 bits.
// Either way the value is that of the float64 expression.
__device__ __forceinline__ double round_sum(long long h, int sh, long long l) {
  const long long lim = 1ll << (62 - sh);
  if (h > -lim && h < lim)
    return __ll2double_rn(static_cast<long long>(static_cast<unsigned long long>(h) << sh) + l);
  return round_exact(h, sh, l, 0);
}

// x 2^e for a finite double: exponent arithmetic when the result stays normal,
// ldexp otherwise (identical results: scaling by a power of two is exact).
__device__ __forceinline__ double scale_pow2(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  const int En = E + e;
  if (E != 0 && E != 0x7ff && En > 0 && En < 0x7ff) return __longlong_as_double(b + (static_cast<long long>(e) << 52));
  return ldexp(x, e);
}

// Shared-memory matrix descriptor: K-major operand tile, rows of 128 bytes,
// 128-byte swizzle, 8-row groups 1024 bytes apart (tile base 1024-aligned).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);  // start address
  d |= static_cast<uint64_t>(1) << 16;                  // leading byte offset (unused for this layout)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;          // stride byte offset: 8 rows
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                  // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::f16: fp32 D, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
// Instruction descriptor, kind::f8f6f4: fp32 D, E4M3 A and B (format 0), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// bounded wait; false on timeout or when another role aborted. CLUSTER: the
// barrier also receives arrivals from the peer CTA (acquire at cluster scope).
template <bool CLUSTER = false>
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                         const TcParams& p) {
  auto try_once = [&]() { return CLUSTER ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity); };
  if (try_once()) return true;
  const uint64_t deadline = globaltimer() + p.timeout_ns;
  for (uint32_t it = 1;; ++it) {
    if (try_once()) return true;
    if ((it & 255u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() > deadline) {
        *abort_flag = 1;
        if (p.err != nullptr) atomicExch(p.err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ int npairs_of(int L, int s) { return min(s, L - 1) - max(1, L - s) + 1; }

// Row blocks of column block c that hold tiles (symmetric: some element with row <= column).
template <int BN, int BM>
__device__ __forceinline__ int rows_of_col(const TcParams& p, int c) {
  return p.sym ? min(p.tiles_m, (BN * (c + 1)) / BM) : p.tiles_m;
}

// Row block bi (BM rows: 128, or 256 for a CTA pair) and column block bj of tile idx.
template <int BN, int BM>
__device__ __forceinline__ void tile_of(const TcParams& p, int idx, int& bi, int& bj) {
  if (p.band_w > 0) {
    const int W = p.band_w, H = p.group_h;
    for (int c0 = 0; c0 < p.tiles_n; c0 += W) {
      const int c1 = min(p.tiles_n, c0 + W);
      const int rmax = rows_of_col<BN, BM>(p, c1 - 1);  // nondecreasing in the column
      for (int r0 = 0; r0 < rmax; r0 += H) {
        const int r1 = min(rmax, r0 + H);
        for (int c = c0; c < c1; ++c) {
          const int k = max(0, min(rows_of_col<BN, BM>(p, c), r1) - r0);
          if (idx < k) {
            bi = r0 + idx;
            bj = c;
            return;
          }
          idx -= k;
        }
      }
    }
    bi = bj = 0;  // not reached for idx < ntiles
    return;
  }
  if (!p.sym) {
    bj = idx / p.tiles_m;  // column-block major: CTAs running together share B blocks
    bi = idx % p.tiles_m;
    return;
  }
  bj = 0;
  for (;;) {
    const int cnt = min(p.tiles_m, (BN * (bj + 1)) / BM);
    if (idx < cnt) break;
    idx -= cnt;
    ++bj;
  }
  bi = idx;
}

// Everything one output tile needs: operands, sizes and the output step.
struct Job {
  const CUtensorMap* ta;
  const CUtensorMap* tb;
  int64_t m0, n0, rows_a, rows_b, m, n;
  int s, KT;
  const int32_t* ea;
  const int32_t* eb;
  bool skip, sym;
  EpiArgs epi;
};

// PAIR: tile is a 256-row pair tile and this CTA (rank 0 or 1) takes rows
// 128 rank .. 128 rank + 127 of it.
template <int BN, bool PAIR = false>
__device__ __forceinline__ Job job_of(const TcParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, int tile,
                                      uint32_t rank = 0) {
  Job j;
  if (p.mats == nullptr) {
    int bi, bj;
    tile_of<BN, PAIR ? 2 * TC_BM : TC_BM>(p, tile, bi, bj);
    j.ta = tmA;
    j.tb = tmB;
    j.m0 = static_cast<int64_t>(bi) * (PAIR ? 2 * TC_BM : TC_BM) + TC_BM * static_cast<int64_t>(rank);
    j.n0 = static_cast<int64_t>(bj) * BN;
    j.rows_a = p.rows_a;
    j.rows_b = p.rows_b;
    j.m = p.m;
    j.n = p.n;
    j.s = p.s;
    j.KT = p.KT;
    j.ea = p.ea;
    j.eb = p.eb;
    j.skip = false;
    j.sym = p.sym != 0;
    j.epi = p.epi;
    return j;
  }
  const int4 t = p.tiles[tile];
  const BatchMat& M = p.mats[t.x];
  // row block t.y of 128 rows, or of 256 for a CTA pair (this CTA: half `rank`)
  j.m0 = static_cast<int64_t>(t.y) * (PAIR ? 2 * TC_BM : TC_BM) + TC_BM * static_cast<int64_t>(rank);
  j.n0 = static_cast<int64_t>(t.z) * BN;
  j.rows_a = M.n_pad;
  j.rows_b = M.n_pad;
  j.m = M.n;
  j.n = M.n;
  j.s = M.s;
  j.KT = static_cast<int>(M.k_pad / (p.beta == 5 ? 128 : TC_BK));  // K atoms of 128 bytes
  j.skip = M.state->done != 0;
  j.sym = true;
  j.ta = &M.tmPa;
  j.ea = M.expsP;
  j.epi.state = M.state;
  j.epi.levels = nullptr;
  j.epi.round32 = 0;
  if (p.phase == 0) {
    j.tb = &M.tmPb;
    j.eb = M.expsP;
    j.epi.kind = EPI_SYM_STORE;
    j.epi.C = M.X2;
    j.epi.ldc = M.n;
    j.epi.P = nullptr;
    j.epi.X2 = nullptr;
    j.epi.ldp = M.n;
    j.epi.ldx = M.n;
  } else {
    j.tb = &M.tmXb;
    j.eb = M.expsX;
    j.epi.kind = EPI_PM_UPDATE;
    j.epi.P = M.buf[p.cur];
    j.epi.ldp = p.cur == 0 ? M.ldp : M.n;
    j.epi.X2 = M.X2;
    j.epi.ldx = M.n;
    j.epi.C = M.buf[1 - p.cur];
    j.epi.ldc = p.cur == 0 ? M.n : M.ldp;
  }
  return j;
}

// Persistent: one CTA per SM walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// The three roles keep their ring and buffer phases across tiles, so the next
// tile's loads and MMAs overlap the current tile's last fold and output.
//
// PAIR (launched as clusters of two CTAs): the cluster walks 256-row pair
// tiles. Each CTA loads its A rows and its half of the B rows, signalling the
// leader's (rank 0) full barrier; the leader alone issues the cta_group::2
// MMAs and its commits arrive on the stage and accumulator barriers of both
// CTAs; both epilogues release a TMEM buffer on the leader's barrier.
//
// WALK: how the CTAs share the launch's tiles.
//   0  each CTA (pair) takes tiles cta, cta + #CTAs, ... (the single-matrix products)
//   2  each CTA takes the next tile from a counter in global memory (the
//      grouped launches of the batched purification, whose tiles differ in
//      work: listed largest first, taken as CTAs free up); the producer takes
//      the tile and passes its index to the MMA and epilogue warps through a
//      small ring in shared memory
//   1  (split) the launch's tiles fill at most half a wave of CTAs (CTA pairs), so
// they are all cut into units of one exact fp32 chunk and shared out evenly in
// contiguous ranges over every CTA; each range's partial level sums are added
// at L2 into the tiles' shared group sums, and the last contributor to a tile
// writes its output. Integer sums do not depend on the split: the result is
// bit-for-bit that of whole tiles.
template <int BN, bool PAIR, bool F8 = false, int WALK = 0>
__global__ void __launch_bounds__(TC_THREADS, 1)
ozaki_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const TcParams p) {
  using Cfg = TcCfg<BN, PAIR, F8>;
  if (p.done != nullptr && *p.done) return;  // uniform: the whole CTA leaves before any setup
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  uint8_t* barp = smem + Cfg::STAGES * Cfg::STAGE_BYTES;
  const uint32_t bar0 = smem_u32(barp);
  auto full_bar = [&](int st) { return bar0 + 8u * st; };
  auto empty_bar = [&](int st) { return bar0 + 8u * (Cfg::STAGES + st); };
  auto accfull_bar = [&](int b) { return bar0 + 8u * (2 * Cfg::STAGES + b); };
  auto accempty_bar = [&](int b) { return bar0 + 8u * (2 * Cfg::STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * Cfg::STAGES + 4);
  // WALK 2: ring of tile indices from the producer to the MMA and epilogue warps
  auto ring_full = [&](int r) { return bar0 + 8u * (2 * Cfg::STAGES + 5 + r); };
  auto ring_empty = [&](int r) { return bar0 + 8u * (2 * Cfg::STAGES + 5 + kTileRing + r); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(barp + 8 * (2 * Cfg::STAGES + 5 + 2 * kTileRing));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* ring_tile = reinterpret_cast<volatile int*>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  // CTA (or CTA pair) index and count for the persistent tile walk
  const int cta_id = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int cta_stride = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);

  if (threadIdx.x == 0) {
    for (int st = 0; st < Cfg::STAGES; ++st) {
      mbar_init(full_bar(st), 1);
      mbar_init(empty_bar(st), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accfull_bar(b), 1);
      mbar_init(accempty_bar(b), PAIR ? 2 * TC_EPI_WARPS : TC_EPI_WARPS);
    }
    mbar_init(drain_bar, 1);
    if (WALK == 2) {
      for (int r = 0; r < kTileRing; ++r) {
        mbar_init(ring_full(r), 1);
        mbar_init(ring_empty(r), 1 + TC_EPI_WARPS);  // the MMA issuer and every epilogue warp
      }
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0 && p.mats == nullptr) {
    tma_prefetch(&tmA);
    tma_prefetch(&tmB);
  }
  if (warp == 1) {
    if (PAIR) {
      tmem_alloc_pair(smem_u32(tmem_slot), Cfg::TMEM_COLS);  // both CTAs, the same columns
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_slot), Cfg::TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // barriers of both CTAs initialised before any remote use
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int CH = p.CH;

  // WALK 1: this CTA's contiguous range [u_begin, u_end) of the launch's chunk
  // units (p.split_unit_count per tile, all tiles split)
  const int KTS_ = p.KT / Cfg::KSUB;  // stages per slice pair (single-matrix launches)
  const int CHS_ = CH / Cfg::KSUB;    // stages per fp32 chunk
  const int64_t split_units = WALK == 1 ? static_cast<int64_t>(p.ntiles) * p.split_unit_count : 0;
  const int64_t u_begin = split_units * cta_id / cta_stride;
  const int64_t u_end = split_units * (cta_id + 1) / cta_stride;
  // unit u: its tile tt, level L and stage range [kb0, kb1)
  auto split_unit = [&](int64_t u, int& tt, int& L, int& kb0, int& kb1) __attribute__((always_inline)) {
    tt = static_cast<int>(u / p.split_unit_count);
    int w = static_cast<int>(u % p.split_unit_count);
    for (L = p.s + 1; L > 2; --L) {
      const int nkb = npairs_of(L, p.s) * KTS_;
      const int nch = (nkb + CHS_ - 1) / CHS_;
      if (w < nch) break;
      w -= nch;
    }
    const int nkb = npairs_of(L, p.s) * KTS_;
    kb0 = w * CHS_;
    kb1 = min(kb0 + CHS_, nkb);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      // for the abort drain: stages ever armed, and the parity of the phase each
      // was last armed in (that phase completes when its copies have landed)
      uint32_t armed = 0, armed_par = 0;
      bool withheld = false;  // stall test: the first stage has been withheld
      // PAIR: both CTAs' copies complete on the leader's full barrier, which expects both
      const uint32_t full_target0 = PAIR ? map_to_cta(full_bar(0), 0) : full_bar(0);
      const uint32_t expect_bytes = PAIR ? 2u * Cfg::STAGE_BYTES : static_cast<uint32_t>(Cfg::STAGE_BYTES);
      const int b_off = PAIR ? static_cast<int>(rank) * (BN / 2) : 0;  // this CTA's half of the B rows
      // one stage: slice pair (i, j), K atoms kt .. kt + KSUB - 1
      auto put_stage = [&](const Job& jb, int i, int j, int kt) __attribute__((always_inline)) -> bool {
        if (!wait_bar<PAIR>(empty_bar(stage), phase ^ 1u, abort_flag, p)) return false;
        const int ya = static_cast<int>((i - 1) * jb.rows_a + jb.m0);
        const int yb = static_cast<int>((j - 1) * jb.rows_b + jb.n0) + b_off;
        const uint32_t sa = sbase + stage * Cfg::STAGE_BYTES;
        if (p.stall_test && !withheld) {
          // stall test: neither the expected bytes nor the copies of this CTA's
          // first stage are issued, so its full barrier never completes and
          // the MMA issuer's bounded wait on it runs out (nothing is in
          // flight for this stage; the later stages drain as in any abort)
          withheld = true;
        } else {
          if (PAIR) {
            const uint32_t fb = full_target0 + 8u * stage;
            if (leader) mbar_arrive_expect_tx(full_bar(stage), expect_bytes);
#pragma unroll
            for (int u = 0; u < Cfg::KSUB; ++u) {
              tma_load_2d_pair(sa + u * Cfg::A_ATOM, jb.ta, fb, (kt + u) * Cfg::ATOM_K, ya);
              tma_load_2d_pair(sa + Cfg::A_BYTES + u * Cfg::B_ATOM, jb.tb, fb, (kt + u) * Cfg::ATOM_K, yb);
            }
          } else {
            mbar_arrive_expect_tx(full_bar(stage), expect_bytes);
            tma_load_2d(sa, jb.ta, full_bar(stage), kt * Cfg::ATOM_K, ya);
            tma_load_2d(sa + Cfg::A_BYTES, jb.tb, full_bar(stage), kt * Cfg::ATOM_K, yb);
          }
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
        }
        if (++stage == Cfg::STAGES) {
          stage = 0;
          phase ^= 1u;
        }
        return true;
      };
      // every stage of one whole tile
      auto put_tile = [&](const Job& jb) __attribute__((always_inline)) {
        const int s = jb.s;
        for (int L = s + 1; L >= 2 && ok; --L) {
          const int i_lo = max(1, L - s), i_hi = min(s, L - 1);
          for (int i = i_lo; i <= i_hi && ok; ++i)
            for (int kt = 0; kt < jb.KT && ok; kt += Cfg::KSUB) ok = put_stage(jb, i, L - i, kt);
        }
      };
      if constexpr (WALK == 0) {
        for (int tile = cta_id; tile < p.ntiles && ok; tile += cta_stride) {
          const Job jb = job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank);
          if (jb.skip) continue;
          put_tile(jb);
        }
      } else if constexpr (WALK == 2) {
        // take tiles from the global counter (skipping finished matrices) and
        // announce each, then -1, to the other warps through the ring
        int rslot = 0;
        uint32_t rph = 0;
        while (ok) {
          int tile = atomicAdd(p.tile_counter, 1);
          while (tile < p.ntiles && job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank).skip) tile = atomicAdd(p.tile_counter, 1);
          if (tile >= p.ntiles) tile = -1;
          if (!wait_bar<false>(ring_empty(rslot), rph ^ 1u, abort_flag, p)) {
            ok = false;
            break;
          }
          ring_tile[rslot] = tile;
          mbar_arrive(ring_full(rslot));  // release: the index is visible to the waiting warps
          if (++rslot == kTileRing) {
            rslot = 0;
            rph ^= 1u;
          }
          if (tile < 0) break;
          put_tile(job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank));
        }
      } else {
        for (int64_t u = u_begin; u < u_end && ok; ++u) {
          int tt, L, kb0, kb1;
          split_unit(u, tt, L, kb0, kb1);
          const Job jb = job_of<BN, PAIR>(p, &tmA, &tmB, tt, rank);
          const int i_lo = max(1, L - p.s);
          for (int kb = kb0; kb < kb1 && ok; ++kb) {
            const int i = i_lo + kb / KTS_;
            ok = put_stage(jb, i, L - i, (kb % KTS_) * Cfg::KSUB);
          }
        }
      }
      if (!ok && leader) {
        // let copies already issued land before shared memory is released (the
        // leader's full barriers count both CTAs' copies)
        for (int st = 0; st < Cfg::STAGES; ++st) {
          if (armed & (1u << st)) {
            const uint32_t par = (armed_par >> st) & 1u;
            const uint64_t dl = globaltimer() + 100000000ull;
            while (!mbar_try_wait(full_bar(st), par) && globaltimer() < dl) {
            }
          }
        }
      }
      if (PAIR && ok) {
        // the leader's commits arrive on this CTA's empty barriers: wait until
        // every stage is released, so no arrival is left in flight at exit
        for (int i = 0; i < Cfg::STAGES && ok; ++i) {
          ok = wait_bar<PAIR>(empty_bar(stage), phase ^ 1u, abort_flag, p);
          if (++stage == Cfg::STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && leader) {
      constexpr uint32_t idesc =
          F8 ? idesc_e4m3(PAIR ? 2 * TC_BM : TC_BM, BN) : idesc_bf16(PAIR ? 2 * TC_BM : TC_BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t aph[2] = {0u, 0u};
      bool ok = true;
      bool issued = false;
      // one stage of MMAs; `first` starts a chunk (waits for a free TMEM buffer
      // and overwrites it), `last` ends it (publishes the buffer)
      auto mma_stage = [&](bool first, bool last) __attribute__((always_inline)) -> bool {
        if (first) {
          if (!wait_bar<PAIR>(accempty_bar(buf), aph[buf] ^ 1u, abort_flag, p)) return false;
          tc_fence_after();
        }
        if (!wait_bar<PAIR>(full_bar(stage), phase, abort_flag, p)) return false;
        tc_fence_after();
        const uint32_t sa = sbase + stage * Cfg::STAGE_BYTES;
        const uint32_t d = tmem + static_cast<uint32_t>(buf * BN);
#pragma unroll
        for (int u = 0; u < Cfg::KSUB; ++u) {
          const uint64_t ad = sdesc_sw128(sa + u * Cfg::A_ATOM);
          const uint64_t bd = sdesc_sw128(sa + Cfg::A_BYTES + u * Cfg::B_ATOM);
#pragma unroll
          for (int ks = 0; ks < TC_MMA_PER_ATOM; ++ks) {
            // advance 32 bytes (16 bf16 or 32 e4m3) along K inside the swizzled row
            const uint32_t acc = (first && u == 0 && ks == 0) ? 0u : 1u;
            if (F8) {
              if (PAIR) {
                umma_e4m3_pair(d, ad + 2ull * ks, bd + 2ull * ks, idesc, acc);
              } else {
                umma_e4m3(d, ad + 2ull * ks, bd + 2ull * ks, idesc, acc);
              }
            } else if (PAIR) {
              umma_bf16_pair(d, ad + 2ull * ks, bd + 2ull * ks, idesc, acc);
            } else {
              umma_bf16(d, ad + 2ull * ks, bd + 2ull * ks, idesc, acc);
            }
          }
        }
        issued = true;
        if (PAIR) {
          umma_commit_pair_both(empty_bar(stage));
        } else {
          umma_commit(empty_bar(stage));
        }
        if (last) {
          if (PAIR) {
            umma_commit_pair_both(accfull_bar(buf));
          } else {
            umma_commit(accfull_bar(buf));
          }
          aph[buf] ^= 1u;
          buf ^= 1;
        }
        if (++stage == Cfg::STAGES) {
          stage = 0;
          phase ^= 1u;
        }
        return true;
      };
      // every stage of one whole tile
      auto mma_tile = [&](const Job& jb) __attribute__((always_inline)) {
        const int s = jb.s;
        // stages per level and per fp32 chunk (KT and CH are multiples of KSUB)
        const int CHS = CH / Cfg::KSUB;
        for (int L = s + 1; L >= 2 && ok; --L) {
          const int nkb = npairs_of(L, s) * (jb.KT / Cfg::KSUB);
          for (int kb = 0; kb < nkb && ok; ++kb) {
            const int kc = kb % CHS;
            ok = mma_stage(kc == 0, (kc == CHS - 1) || (kb == nkb - 1));
          }
        }
      };
      if constexpr (WALK == 0) {
        for (int tile = cta_id; tile < p.ntiles && ok; tile += cta_stride) {
          const Job jb = job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank);
          if (jb.skip) continue;
          mma_tile(jb);
        }
      } else if constexpr (WALK == 2) {
        int rslot = 0;
        uint32_t rph = 0;
        while (ok) {
          if (!wait_bar<false>(ring_full(rslot), rph, abort_flag, p)) {
            ok = false;
            break;
          }
          const int tile = ring_tile[rslot];
          mbar_arrive(ring_empty(rslot));
          if (++rslot == kTileRing) {
            rslot = 0;
            rph ^= 1u;
          }
          if (tile < 0) break;
          mma_tile(job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank));
        }
      } else {
        for (int64_t u = u_begin; u < u_end && ok; ++u) {
          int tt, L, kb0, kb1;
          split_unit(u, tt, L, kb0, kb1);
          for (int kb = kb0; kb < kb1 && ok; ++kb) ok = mma_stage(kb == kb0, kb == kb1 - 1);
        }
      }
      if (!ok && issued) {
        // wait for the MMAs in flight before TMEM is released
        if (PAIR) {
          umma_commit_pair_self(drain_bar);
        } else {
          umma_commit(drain_bar);
        }
        const uint64_t dl = globaltimer() + 100000000ull;
        while (!mbar_try_wait(drain_bar, 0) && globaltimer() < dl) {
        }
      }
      if (PAIR && ok) {
        // both epilogues arrive on this CTA's accumulator barriers: wait for
        // their last releases, so no arrival is left in flight at exit
        for (int b = 0; b < 2 && ok; ++b) ok = wait_bar<PAIR>(accempty_bar(b), aph[b] ^ 1u, abort_flag, p);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int COLS = Cfg::COLS;
    const int e = warp - 2;
    const int q = warp & 3;   // TMEM lane quadrant this warp may access
    const int h = e >> 2;     // which half of the BN columns
    const int row = 32 * q + lane;
    const int cbase = h * COLS;
    const uint32_t taddr_row = tmem + (static_cast<uint32_t>(32 * q) << 16);
    // fold buffers of this thread (whole tiles): the int64 group sums, or the
    // running group and the float64 sum D; element c at [32 c] (a warp touches
    // 256 contiguous bytes per column), private to this CTA and L2-resident
    long long* scr_i = reinterpret_cast<long long*>(p.scratch) +
                       static_cast<int64_t>(blockIdx.x) * (2 * TC_BM * BN) + e * (COLS * 32) + lane;
    long long* scr_d = scr_i + TC_BM * BN;
    // WALK 1: the group sums of (tile tt, this CTA's row half), shared by the
    // CTAs that contribute to the tile; same element layout
    auto split_area_of = [&](int tt, int gidx) __attribute__((always_inline)) -> long long* {
      return p.split_area + ((static_cast<int64_t>(tt) * (PAIR ? 2 : 1) + rank) * 2 + gidx) * (TC_BM * BN) +
             e * (COLS * 32) + lane;
    };

    int32_t S[COLS];
    int buf = 0;
    uint32_t aph[2] = {0u, 0u};
    bool ok = true;
    // PAIR: TMEM buffers are released on the leader's barrier
    const uint32_t accempty_target0 = PAIR ? map_to_cta(accempty_bar(0), 0) : accempty_bar(0);

    // one finished chunk from TMEM added into the level sum S (one call site
    // per kernel: a second, specialised copy costs the register allocator far
    // more than zeroing S)
    auto drain_chunk = [&]() __attribute__((always_inline)) -> bool {
      // one lane polls the barrier (32 pollers per warp would crowd the
      // barrier word the MMA issuer and the copies also use); the warp then
      // synchronises and orders its TMEM loads after that wait (tcgen05.ld
      // below is warp-collective, so the whole warp takes the same branch)
      int got = 0;
      if (lane == 0) got = wait_bar<PAIR>(accfull_bar(buf), aph[buf], abort_flag, p) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) return false;
      tc_fence_after();
#pragma unroll
      for (int g = 0; g < COLS / 16; ++g) {
        uint32_t v[16];
        tmem_ld16(taddr_row + static_cast<uint32_t>(buf * BN + cbase + 16 * g), v);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) S[16 * g + t] += __float2int_rn(__uint_as_float(v[t]));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (PAIR) {
          mbar_arrive_cluster(accempty_target0 + 8u * buf);
        } else {
          mbar_arrive(accempty_bar(buf));
        }
      }
      aph[buf] ^= 1u;
      buf ^= 1;
      return true;
    };

    // the output step of a finished tile: unscale the group sums in a0 (group 0)
    // and a1 (group 1, or D with three or more groups) and write C (or the
    // update). The group sums are read from L2 (.cg): reductions at L2, and for
    // the split those of other CTAs, never pass through this SM's L1.
    auto output_tile = [&](const Job& jb, int64_t m0, int64_t n0, int s, const long long* a0,
                           const long long* a1) __attribute__((always_inline)) {
      const int64_t r = m0 + row;
      if (r >= jb.m) return;
      const int32_t er = jb.ea[r];
      const bool upd = jb.epi.kind == EPI_PM_UPDATE;
      const double wa = upd ? jb.epi.state->alpha : 0.0;
      const double w2 = upd ? jb.epi.state->b2 : 0.0;
      const double w3 = upd ? jb.epi.state->b3 : 0.0;
      // last group (levels 2 .. L_a, L_a = 2 + (s - 1) mod G) in a0, or in a1
      // for two groups (then a0 holds group 0, weight 2^(-beta (s+1))); with
      // three or more groups the earlier ones are summed in D (a1)
      const double lscale = ldexp(1.0, -p.beta * (2 + (s - 1) % p.group));
      const bool has_d = s > p.group;
      const bool two_groups = has_d && s <= 2 * p.group;
      // weight of the rounded sum: 2^(-beta (s+1)) for two groups, 2^(-beta L_a)
      // for one, none with D (already scaled)
      const int e_acc = two_groups ? -p.beta * (s + 1) : (has_d ? 0 : -p.beta * (2 + (s - 1) % p.group));
      const uint64_t pol = policy_evict_last();
      double* Cout = jb.epi.C;
      const int64_t ldc = jb.epi.ldc;
      // batches of 8 columns: issue every load of the batch, then compute and
      // store; the next batch's P and P^2 lines are requested into L1 meanwhile
      auto prefetch_batch = [&](int gb) __attribute__((always_inline)) {
        const int64_t c0 = n0 + cbase + 8 * gb;
        if (!upd || gb >= COLS / 8 || c0 >= jb.n) return;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (c0 + t < jb.n) {
            prefetch_l1(jb.epi.P + (c0 + t) * jb.epi.ldp + r);
            prefetch_l1(jb.epi.X2 + (c0 + t) * jb.epi.ldx + r);
          }
        }
      };
      for (int g = 0; g < COLS / 8; ++g) {
        const int64_t col0 = n0 + cbase + 8 * g;
        if (col0 >= jb.n) break;
        long long ti[8], td[8];
        double pv[8], xv[8];
        int32_t ecv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int c = 8 * g + t;
          const int64_t col = col0 + t;
          const bool ok = col < jb.n;
          ti[t] = ld_l2(a0 + 32 * c, pol);
          td[t] = has_d ? ld_l2(a1 + 32 * c, pol) : 0ll;
          ecv[t] = ok ? jb.eb[col] : 0;
          // P and P^2 are exactly symmetric: read them at (col, r), coalesced across the warp
          pv[t] = (upd && ok) ? jb.epi.P[col * jb.epi.ldp + r] : 0.0;
          xv[t] = (upd && ok) ? jb.epi.X2[col * jb.epi.ldx + r] : 0.0;
        }
        prefetch_batch(g + 1);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int64_t col = col0 + t;
          if (col >= jb.n) break;
          if (jb.sym && r > col) continue;  // the (col, r) element's mirror covers it
          // one or two groups: the exact integer combination rounded once and
          // scaled by 2^e_acc (exact); three or more: the float64 sum D of the
          // earlier groups plus the last
          const double acc = two_groups ? round_sum(td[t], p.beta * p.group, ti[t])
                                        : (has_d ? __longlong_as_double(td[t]) + static_cast<double>(ti[t]) * lscale
                                                 : static_cast<double>(ti[t]));
          double v = (er == kBadExp || ecv[t] == kBadExp) ? __longlong_as_double(0x7ff8000000000000ll)
                                                          : scale_pow2(acc, er + ecv[t] + e_acc);
          if (upd) v = wa * pv[t] + w2 * xv[t] + w3 * v;
          v = stored_value(v, jb.epi.round32 != 0);
          Cout[r * ldc + col] = v;
          if (jb.sym && r < col) Cout[col * ldc + r] = v;
        }
      }
    };

    if constexpr (WALK != 1) {
      // ---- whole tiles: cta, cta + #CTAs, ... (WALK 0) or as the producer
      // announces them through the ring (WALK 2)
      int rslot = 0;
      uint32_t rph = 0;
      for (int tile = cta_id - cta_stride; ok;) {
        if constexpr (WALK == 0) {
          tile += cta_stride;
          if (tile >= p.ntiles) break;
        } else {
          int got = 0, t = 0;
          if (lane == 0) {
            got = wait_bar<false>(ring_full(rslot), rph, abort_flag, p) ? 1 : 0;
            if (got) {
              t = ring_tile[rslot];
              mbar_arrive(ring_empty(rslot));
            }
          }
          got = __shfl_sync(0xffffffffu, got, 0);
          t = __shfl_sync(0xffffffffu, t, 0);
          if (++rslot == kTileRing) {
            rslot = 0;
            rph ^= 1u;
          }
          if (!got) {
            ok = false;
            break;
          }
          if (t < 0) break;
          tile = t;
        }
        int64_t m0, n0;
        int s, KT;
        bool skip;
        {
          const Job jb = job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank);
          m0 = jb.m0;
          n0 = jb.n0;
          s = jb.s;
          KT = jb.KT;
          skip = jb.skip;
        }
        if (skip) continue;
        for (int L = s + 1; L >= 2 && ok; --L) {
#pragma unroll
          for (int c = 0; c < COLS; ++c) S[c] = 0;
          if (L == 2 && p.epi.kind == EPI_PM_UPDATE && p.mats == nullptr && m0 + row < p.m) {
            // the update reads P and P^2 in the output pass: ask L2 for this
            // thread's elements while the last level's chunks are still running
            for (int c = 0; c < COLS; ++c) {
              const int64_t col = n0 + cbase + c;
              if (col >= p.n) break;
              prefetch_l2(p.epi.P + col * p.epi.ldp + m0 + row);
              prefetch_l2(p.epi.X2 + col * p.epi.ldx + m0 + row);
            }
          }
          const int nkb = npairs_of(L, s) * KT;
          const int nch = (nkb + CH - 1) / CH;
          for (int ch = 0; ch < nch && ok; ++ch) ok = drain_chunk();
          if (!ok) break;
          if (p.epi.kind == EPI_LEVELS && p.mats == nullptr) {
            // test hook: write the exact level sum itself
            const int64_t r = m0 + row;
            if (r < p.m) {
#pragma unroll
              for (int c = 0; c < COLS; ++c) {
                const int64_t col = n0 + cbase + c;
                if (col < p.n) p.epi.levels[static_cast<int64_t>(L - 2) * p.m * p.n + r * p.n + col] = S[c];
              }
            }
            continue;
          }
          // ---- fold the exact level sum (groups of levels, smallest first; see the header)
          {
            const uint64_t pol = policy_evict_last();
            // up to G consecutive levels (G = 4 for beta 7 and 5, 3 for beta 8)
            // combine exactly in int64, T = sum S_L 2^(beta (L_a - L)) < 2^53; the
            // first level of a group stores its sum, the others add theirs at L2
            // (red: nothing comes back, so the fold costs no round trip). With at
            // most two groups each has its own area (group 0 in scr_i, group 1 in
            // scr_d) and both are finished by the output pass. With three or more,
            // scr_i holds the running group: at the end of a group (other than the
            // last) its exact value T 2^(-beta L_a) is read back and added to D
            // (scr_d) in float64.
            const int G = p.group;
            const int gpos = (s + 1 - L) % G;
            const int gidx = (s + 1 - L) / G;
            const bool two_areas = s <= 2 * G;
            long long* area = (two_areas && gidx == 1) ? scr_d : scr_i;
            const bool gend = !two_areas && (gpos == G - 1) && (L != 2);
            const int La = L + gpos;
            const bool first_group = gidx == 0;
            const double gscale = ldexp(1.0, -p.beta * La);
            const long long wgt = 1ll << (p.beta * gpos);
            if (!gend) {
#pragma unroll
              for (int c = 0; c < COLS; ++c) {
                const long long v = static_cast<long long>(S[c]) * wgt;
                if (gpos == 0) {
                  st_keep(area + 32 * c, v, pol);
                } else {
                  red_add_keep(area + 32 * c, v, pol);
                }
              }
            } else {
#pragma unroll
              for (int g = 0; g < COLS / 8; ++g) {
                long long told[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) told[t] = ld_l2(scr_i + 32 * (8 * g + t), pol);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                  const int c = 8 * g + t;
                  const long long T = told[t] + static_cast<long long>(S[c]) * wgt;
                  const double gv = static_cast<double>(T) * gscale;
                  const double d = first_group ? gv : __longlong_as_double(ld_l2(scr_d + 32 * c, pol)) + gv;
                  st_keep(scr_d + 32 * c, __double_as_longlong(d), pol);
                }
              }
            }
          }
          if (L != 2) continue;
          // ---- last level: unscale and apply the output step
          const Job jb = job_of<BN, PAIR>(p, &tmA, &tmB, tile, rank);
          output_tile(jb, m0, n0, s, scr_i, scr_d);
        }
      }
    } else if (u_begin < u_end) {
      // ---- the split: (tile, level) runs of this CTA's range, each drained
      // into S and added at L2 to the tile's group sums (at most two groups,
      // areas zeroed before the launch); leaving a tile counts this warp in
      // for it, and the last of the tile's contributors writes this warp's
      // part of the output
      const uint64_t pol = policy_evict_last();
      const int s = p.s;
      const int G = p.group;
      const int64_t units_per_tile = p.split_unit_count;
      // CTA (pair) that owns unit u
      auto owner = [&](int64_t u) __attribute__((always_inline)) -> int64_t {
        return ((u + 1) * cta_stride + split_units - 1) / split_units - 1;
      };
      // tiles whose output this warp writes, after its whole range (a range
      // shorter than a tile meets at most two tiles)
      int out_tiles[2] = {-1, -1};
      int n_out = 0;
      // the tiles this range meets, level by level as whole tiles are walked;
      // level L of tile tt holds units [base, base + nch_L) of the launch
      const int tt_lo = static_cast<int>(u_begin / units_per_tile);
      const int tt_hi = static_cast<int>((u_end - 1) / units_per_tile);
      for (int tt = tt_lo; tt <= tt_hi && ok; ++tt) {
        int base = static_cast<int>(static_cast<int64_t>(tt) * units_per_tile);
        for (int L = s + 1; L >= 2 && ok; --L) {
          const int nch_l = (npairs_of(L, s) * KTS_ + CHS_ - 1) / CHS_;
          const int lo = max(base, static_cast<int>(u_begin));
          const int hi = min(base + nch_l, static_cast<int>(u_end));
          base += nch_l;
          if (lo >= hi) continue;
#pragma unroll
          for (int c = 0; c < COLS; ++c) S[c] = 0;
          for (int ch = lo; ch < hi && ok; ++ch) ok = drain_chunk();
          if (!ok) break;
          const int gpos = (s + 1 - L) % G;
          long long* area = split_area_of(tt, (s + 1 - L) / G);
          const long long wgt = 1ll << (p.beta * gpos);
#pragma unroll
          for (int c = 0; c < COLS; ++c) red_add_keep(area + 32 * c, static_cast<long long>(S[c]) * wgt, pol);
        }
        if (!ok) break;
        __threadfence();  // this lane's reductions before the count
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          // the CTAs (pairs) whose non-empty ranges meet this tile (with fewer
          // units than CTAs some ranges are empty)
          const int64_t u0 = static_cast<int64_t>(tt) * units_per_tile;
          int contributors = 0;
          for (int64_t c = owner(u0); c <= owner(u0 + units_per_tile - 1); ++c)
            contributors += (split_units * (c + 1) / cta_stride > split_units * c / cta_stride) ? 1 : 0;
          int* cnt = p.split_cnt + (static_cast<int64_t>(tt) * (PAIR ? 2 : 1) + rank) * TC_EPI_WARPS + e;
          last = atomicAdd(cnt, 1) == contributors - 1 ? 1 : 0;
        }
        if (__shfl_sync(0xffffffffu, last, 0) != 0 && n_out < 2) out_tiles[n_out++] = tt;
      }
      if (ok && n_out > 0) {
        __threadfence();  // every contributor's reductions before the reads
        for (int k = 0; k < n_out; ++k) {
          const Job jb = job_of<BN, PAIR>(p, &tmA, &tmB, out_tiles[k], rank);
          output_tile(jb, jb.m0, jb.n0, s, split_area_of(out_tiles[k], 0), split_area_of(out_tiles[k], 1));
        }
      }
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // neither CTA leaves while the other may still use its barriers or TMEM
  if (warp == 1) {
    tc_fence_after();
    if (PAIR) {
      tmem_dealloc_pair(tmem, Cfg::TMEM_COLS);
    } else {
      tmem_dealloc(tmem, Cfg::TMEM_COLS);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// 2-D view of s stacked digit planes (bf16, or E4M3 bytes when f8): dim0 = k_pad
// (contiguous), dim1 = s * rows; boxes of one 128-byte row by box_rows.
bool make_plane_map(CUtensorMap* tm, const void* planes, int64_t k_pad, int64_t rows_total, int box_rows,
                    bool f8 = false) {
  auto fn = encode_fn();
  if (fn == nullptr) return false;
  const int eb = f8 ? 1 : 2;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(k_pad), static_cast<cuuint64_t>(rows_total)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(k_pad * eb)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(TC_ROW_BYTES / eb), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(planes), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool make_plane_map_ext(CUtensorMap* tm, const void* planes, int64_t k_pad, int64_t rows_total, int box_rows,
                        bool f8) {
  return make_plane_map(tm, planes, k_pad, rows_total, box_rows, f8);
}

namespace {

// Set before every launch rather than once per process: the attribute belongs
// to the kernel as loaded in the current context, and a context created anew
// (after cudaDeviceReset) starts from the default limit. The call is host-side
// only and costs about a microsecond against milliseconds of kernel.
template <int BN, bool PAIR, bool F8 = false, int WALK = 0>
cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(ozaki_tc_kernel<BN, PAIR, F8, WALK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<BN, PAIR, F8>::SMEM);
}

template <int BN, bool PAIR = false, bool F8 = false, int WALK = 0>
cudaError_t launch_tc_impl(const CUtensorMap& ta, const CUtensorMap& tb, const TcParams& p, int grid,
                           cudaStream_t st) {
  using Cfg = TcCfg<BN, PAIR, F8>;
  cudaError_t e = set_smem_attr<BN, PAIR, F8, WALK>();
  if (e != cudaSuccess) return e;
  if (PAIR) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, ozaki_tc_kernel<BN, PAIR, F8, WALK>, ta, tb, p);
    if (e != cudaSuccess) return e;
  } else {
    ozaki_tc_kernel<BN, PAIR, F8, WALK><<<grid, TC_THREADS, Cfg::SMEM, st>>>(ta, tb, p);
  }
  count_launch();
  return cudaGetLastError();
}

bool g_pairing = true;

// One-shot stall test (dmp_test_stall_next_product): wait limit in microseconds
// for the next tcgen05 product launch, 0 = off.
std::atomic<int> g_stall_us{0};

// CTA pairs of the PAIR kernel that can be resident at once (0: none)
int tc_max_pairs() {
  static int pairs = -1;
  if (pairs < 0) {
    pairs = 0;
    if (set_smem_attr<256, true>() == cudaSuccess) {
      cudaLaunchConfig_t cfg;
      std::memset(&cfg, 0, sizeof(cfg));
      cfg.gridDim = dim3(2);
      cfg.blockDim = dim3(TC_THREADS);
      cfg.dynamicSmemBytes = TcCfg<256, true>::SMEM;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int c = 0;
      if (cudaOccupancyMaxActiveClusters(&c, ozaki_tc_kernel<256, true>, &cfg) == cudaSuccess) pairs = c;
    }
    (void)cudaGetLastError();
    pairs = std::min(pairs, kTcMaxCtas / 2);
  }
  return pairs;
}

}  // namespace

bool tc_pairs_available() { return g_pairing && tc_max_pairs() > 0; }

int set_stall_test(int wait_limit_us) {
  if (wait_limit_us < 0) return DMP_ERR_INVALID_ARG;
  g_stall_us.store(wait_limit_us);
  return DMP_OK;
}

int set_tc_pairing(int enable) {
  const int prev = g_pairing ? 1 : 0;
  g_pairing = enable != 0;
  return prev;
}

int tc_max_ctas() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return std::min(sms, kTcMaxCtas);
}

size_t tc_scratch_bytes() { return static_cast<size_t>(kTcMaxCtas) * 2 * TC_BM * 256 * sizeof(double); }

// Split launches: fewer than kTcMaxCtas / 2 tiles of one CTA (or kTcMaxCtas / 4
// of a CTA pair, two row halves each), each with two TC_BM x 256 int64 group
// sums per CTA, then one counter per (tile, CTA, epilogue warp).
static size_t tc_split_area_bytes() {
  return static_cast<size_t>(kTcMaxCtas / 2) * 2 * TC_BM * 256 * sizeof(long long);
}
size_t tc_split_bytes() {
  return tc_split_area_bytes() + static_cast<size_t>(kTcMaxCtas / 2) * TC_EPI_WARPS * sizeof(int);
}

bool g_split_tiles = true;

int set_tc_split_tiles(int enable) {
  const int prev = g_split_tiles ? 1 : 0;
  g_split_tiles = enable != 0;
  return prev;
}

cudaError_t launch_ozaki_tc(const void* A, const void* B, const int32_t* ea, const int32_t* eb, int64_t m,
                            int64_t n, int64_t rows_a, int64_t rows_b, int64_t k_pad, int s, int beta, int sym,
                            const EpiArgs& epi, const int* done, int* err, double* scratch, void* split_ws,
                            cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const bool f8 = beta == 5;  // E4M3 nearest digits
  const int BN = 256;
  const int atom_k = f8 ? 128 : TC_BK;
  if (rows_a % TC_BM != 0 || rows_b % BN != 0 || k_pad % atom_k != 0) return cudaErrorInvalidValue;
  // products run on CTA pairs (256 x 256 tiles, 2-SM MMA) when rows allow
  const bool pair = g_pairing && rows_a % (2 * TC_BM) == 0 && k_pad % (2 * atom_k) == 0 && tc_max_pairs() > 0;
  const int BM = pair ? 2 * TC_BM : TC_BM;
  CUtensorMap ta, tb;
  if (!make_plane_map(&ta, A, k_pad, static_cast<int64_t>(s) * rows_a, TC_BM, f8)) return cudaErrorInvalidValue;
  if (!make_plane_map(&tb, B, k_pad, static_cast<int64_t>(s) * rows_b, pair ? BN / 2 : BN, f8))
    return cudaErrorInvalidValue;
  TcParams p;
  p.mats = nullptr;
  p.tiles = nullptr;
  p.phase = 0;
  p.cur = 0;
  p.s = s;
  p.beta = beta;
  p.KT = static_cast<int>(k_pad / atom_k);
  // K chunk in atoms: 1024 (beta 7: 127^2; beta 8 nearest: 128^2) or 65536
  // (beta 5 nearest: 16^2) K elements keep every fp32 partial sum at most 2^24
  p.CH = f8 ? 512 : 16;
  p.group = beta == 8 ? 3 : 4;
  p.m = m;
  p.n = n;
  p.rows_a = rows_a;
  p.rows_b = rows_b;
  p.sym = sym;
  p.tiles_m = static_cast<int>(rows_a / BM);
  p.tiles_n = static_cast<int>(rows_b / BN);
  {
    // blocks of about as many tiles as run at once, near-square in elements
    const int units = pair ? tc_max_pairs() : tc_max_ctas();
    int w = static_cast<int>(std::lround(std::sqrt(static_cast<double>(units) * BM / BN)));
    w = std::max(1, std::min(w, p.tiles_n));
    p.band_w = w;
    p.group_h = std::max(1, units / w);
  }
  p.ea = ea;
  p.eb = eb;
  p.epi = epi;
  p.done = done;
  p.err = err;
  p.timeout_ns = 5000000000ull;
  p.stall_test = 0;
  // the stall test is taken by a launch that runs now, never by one being
  // captured into a graph (every replay would stall)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
    if (const int us = g_stall_us.exchange(0); us > 0) {
      p.stall_test = 1;
      p.timeout_ns = 1000ull * static_cast<unsigned long long>(us);
    }
  }
  int ntiles = 0;
  if (sym) {
    for (int bj = 0; bj < p.tiles_n; ++bj) ntiles += std::min(p.tiles_m, (BN * (bj + 1)) / BM);
  } else {
    ntiles = p.tiles_m * p.tiles_n;
  }
  p.ntiles = ntiles;
  p.scratch = scratch;
  // split: when the tiles fill at most half a wave of CTAs (CTA pairs), they
  // are all cut into fp32-chunk units shared out evenly over every CTA, so the
  // idle part of the wave works too. Needs at most two level groups (their
  // sums are then finished in the output pass) and the caller's split
  // workspace. Measured on GB300 (INT8, s = 5 with an 8-slice refinement):
  // 10 pair tiles (n = 1024) 0.197 -> 0.117 ms per product, 36 (n = 2048) 0.273
  // -> 0.204 ms, but 66 of 74 pairs (n = 2816) 0.339 -> 0.443 ms: the units'
  // L2 reductions then cost more than the few idle pairs; sharing out only the
  // last partial wave of a larger launch measured slower as well (n >= 4096).
  const int units = pair ? tc_max_pairs() : tc_max_ctas();
  p.split_unit_count = 0;
  p.split_area = nullptr;
  p.split_cnt = nullptr;
  p.tile_counter = nullptr;
  const bool split =
      g_split_tiles && split_ws != nullptr && 2 * ntiles <= units && s <= 2 * p.group && epi.kind != EPI_LEVELS;
  if (split) {
    const int ranks = pair ? 2 : 1;
    const int KSUB = pair ? 2 : 1;
    const int kts = p.KT / KSUB, chs = p.CH / KSUB;
    int cnt = 0;
    for (int L = s + 1; L >= 2; --L) {
      const int np = std::min(s, L - 1) - std::max(1, L - s) + 1;
      cnt += (np * kts + chs - 1) / chs;
    }
    p.split_unit_count = cnt;
    p.split_area = static_cast<long long*>(split_ws);
    p.split_cnt = reinterpret_cast<int*>(static_cast<char*>(split_ws) + tc_split_area_bytes());
    // the tiles' group sums and counters start from zero
    const size_t area = static_cast<size_t>(ntiles) * ranks * 2 * TC_BM * 256 * sizeof(long long);
    cudaError_t e = cudaMemsetAsync(split_ws, 0, area, st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(p.split_cnt, 0, static_cast<size_t>(ntiles) * ranks * TC_EPI_WARPS * sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  ProfScope prof(DMP_PROF_PRODUCT, st);
  const int grid_units = split ? units : std::min(ntiles, units);
  if (pair) {
    const int grid = 2 * grid_units;
    if (split)
      return f8 ? launch_tc_impl<256, true, true, 1>(ta, tb, p, grid, st)
                : launch_tc_impl<256, true, false, 1>(ta, tb, p, grid, st);
    return f8 ? launch_tc_impl<256, true, true>(ta, tb, p, grid, st) : launch_tc_impl<256, true>(ta, tb, p, grid, st);
  }
  const int grid = grid_units;
  if (split)
    return f8 ? launch_tc_impl<256, false, true, 1>(ta, tb, p, grid, st)
              : launch_tc_impl<256, false, false, 1>(ta, tb, p, grid, st);
  return f8 ? launch_tc_impl<256, false, true>(ta, tb, p, grid, st) : launch_tc_impl<256, false>(ta, tb, p, grid, st);
}

cudaError_t launch_ozaki_tc_grouped(const BatchMat* mats, const int4* tiles, int ntiles, int bn, bool pair, int beta,
                                    int phase, int cur, int* err, double* scratch, int* counter, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  p.beta = beta;
  p.CH = beta == 5 ? 512 : 16;
  p.group = beta == 8 ? 3 : 4;
  p.ntiles = ntiles;
  p.scratch = scratch;
  p.sym = 1;
  p.mats = mats;
  p.tiles = tiles;
  p.phase = phase;
  p.cur = cur;
  p.err = err;
  p.done = nullptr;
  p.timeout_ns = 5000000000ull;
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  if (pair) {
    // CTA pairs (256-row tiles, 256 columns): the pairs walk the list (largest
    // matrices first) round robin
    if (bn != 256 || tc_max_pairs() <= 0) return cudaErrorInvalidValue;
    const int grid = 2 * std::min(ntiles, tc_max_pairs());
    ProfScope prof(DMP_PROF_PRODUCT, st);
    return beta == 5 ? launch_tc_impl<256, true, true>(unused, unused, p, grid, st)
                     : launch_tc_impl<256, true, false>(unused, unused, p, grid, st);
  }
  // single CTAs take tiles from a counter as they free up (the tiles differ in
  // work: the list holds the largest matrices' tiles first)
  p.tile_counter = counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int grid = std::min(ntiles, tc_max_ctas());
  ProfScope prof(DMP_PROF_PRODUCT, st);
  if (beta == 5) return bn == 256 ? launch_tc_impl<256, false, true, 2>(unused, unused, p, grid, st)
                                  : cudaErrorInvalidValue;  // E4M3 digits: 256-column tiles
  if (bn == 128) return launch_tc_impl<128, false, false, 2>(unused, unused, p, grid, st);
  return launch_tc_impl<256, false, false, 2>(unused, unused, p, grid, st);
}

}  // namespace dmp
