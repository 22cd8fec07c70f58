// Batched purification: many Hamiltonians of different sizes purified
// together (dm_purify_batched).
//
// Every phase of an iteration is one grouped launch over all matrices -- the
// row split, the tcgen05 product over the upper tiles of every matrix (one
// persistent kernel with per-matrix TMA descriptors in global memory), the
// measures and stopping rules, the split of P^2 and the product with the fused
// update. Matrices that stopped are skipped by every kernel. Two iterations
// (ping-pong between the caller's P and a workspace copy) form the body of a
// CUDA graph WHILE loop whose condition the stopping-rule kernel clears once
// every matrix has stopped, so the whole loop runs as one graph launch with no
// host round trip. Graphs are cached per argument set.
//
// Slice modes: INT8, BF16 (nearest 8-bit digits) and E4M3 (nearest 5-bit
// digits, one-byte planes, 256-column tiles only).
//
// The autotuner picks the tile width (128 or 256 columns) by timing the P^2
// product of the batch with both, and, when opts->slices is 0, the slice count:
// the smallest s whose band energy on the largest matrix agrees with that of
// s + 2 to the target (1e-8 relative, or opts->energy_tol when set). Choices are
// cached per batch shape for the life of the process.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int kMeasBlk = 32;  // measure CTAs per matrix

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-matrix partial measures over the upper triangle (the quantities of the
// single path's measure kernel). Batch rows are short (at most a few thousand
// entries), so each warp takes whole rows: rows blockIdx.x 8 + w, + 8 kMeasBlk,
// ... with the upper entries spread over the lanes, four independent
// accumulator sets per lane, combined in a fixed order (reproducible sums).
__global__ void __launch_bounds__(256)
measure_grouped_kernel(const BatchMat* __restrict__ mats, int cur, double* __restrict__ part) {
  const BatchMat& M = mats[blockIdx.y];
  if (M.state->done) return;
  const int64_t n = M.n;
  const double* P = M.buf[cur];
  const int64_t ldp = cur == 0 ? M.ldp : n;
  const double* X2 = M.X2;
  const double* H = M.H;
  const int64_t ldh = M.ldh;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double a_px[4] = {0.0, 0.0, 0.0, 0.0}, a_id[4] = {0.0, 0.0, 0.0, 0.0}, a_ph[4] = {0.0, 0.0, 0.0, 0.0};
  double d_p = 0.0, d_x = 0.0, d_px = 0.0, d_id = 0.0, d_ph = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * 8 + w; i < n; i += static_cast<int64_t>(gridDim.x) * 8) {
    const double* pr = P + i * ldp;
    const double* xr = X2 + i * n;
    const double* hr = H + i * ldh;
    if (lane == 0) {
      const double p = pr[i], x = xr[i], h = hr[i];
      d_p += p;
      d_x += x;
      d_px += p * x;
      d_id += (x - p) * (x - p);
      d_ph += p * h;
    }
    int64_t j = i + 1 + lane;
    for (; j + 96 < n; j += 128) {
      double pv[4], xv[4], hv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        pv[u] = pr[j + 32 * u];
        xv[u] = xr[j + 32 * u];
        hv[u] = hr[j + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a_px[u] += pv[u] * xv[u];
        a_id[u] += (xv[u] - pv[u]) * (xv[u] - pv[u]);
        a_ph[u] += pv[u] * hv[u];
      }
    }
    for (; j < n; j += 32) {
      const double p = pr[j], x = xr[j], h = hr[j];
      a_px[0] += p * x;
      a_id[0] += (x - p) * (x - p);
      a_ph[0] += p * h;
    }
  }
  const double u_px = (a_px[0] + a_px[1]) + (a_px[2] + a_px[3]);
  const double u_id = (a_id[0] + a_id[1]) + (a_id[2] + a_id[3]);
  const double u_ph = (a_ph[0] + a_ph[1]) + (a_ph[2] + a_ph[3]);
  __shared__ double red[8][8];
  double v[8] = {d_p, d_x, d_px, u_px, d_id, u_id, d_ph, u_ph};
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 8; ++q) red[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < 8) {
    double t = 0.0;
    for (int ww = 0; ww < 8; ++ww) t += red[ww][threadIdx.x];
    part[(static_cast<int64_t>(blockIdx.y) * kMeasBlk + blockIdx.x) * 8 + threadIdx.x] = t;
  }
}

// One thread per matrix applies the stopping rules; the block then tells the
// graph (or, in stream mode, the host through *active) whether any matrix
// still runs.
__global__ void measure_grouped_final_kernel(const BatchMat* __restrict__ mats, int nmats,
                                             const double* __restrict__ part, cudaGraphConditionalHandle cond,
                                             int set_cond, int* __restrict__ active) {
  __shared__ int any_active;
  if (threadIdx.x == 0) any_active = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < nmats; b += blockDim.x) {
    PurifyState* st = mats[b].state;
    if (!st->done) {
      double tot[8];
      for (int q = 0; q < 8; ++q) {
        double t = 0.0;
        for (int k = 0; k < kMeasBlk; ++k) t += part[(static_cast<int64_t>(b) * kMeasBlk + k) * 8 + q];
        tot[q] = t;
      }
      pm_decide(st, tot);
    }
    if (!st->done) atomicOr(&any_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && set_cond) cudaGraphSetConditional(cond, any_active ? 1u : 0u);
  if (threadIdx.x == 0 && active != nullptr) *active = any_active;
}

// The result of a matrix that stopped after an odd number of updates sits in
// the workspace copy: move it to the caller's P.
__global__ void finish_grouped_kernel(const BatchMat* __restrict__ mats) {
  const BatchMat& M = mats[blockIdx.y];
  if ((M.state->iter & 1) == 0) return;
  const int64_t n = M.n;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n * n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    M.buf[0][i * M.ldp + j] = M.buf[1][e];
  }
}

// The refinement step (one McWeeny step P' = 3 P^2 - 2 P^3 with r-slice
// products after the loop, Sec. "Precision Requirements Sweep"): matrices that
// ended without an error run again (done cleared) with the McWeeny weights.
__global__ void refine_begin_kernel(const BatchMat* __restrict__ mats, int nmats) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nmats; b += gridDim.x * blockDim.x) {
    PurifyState* st = mats[b].state;
    if (st->status < 0) continue;
    st->alpha = 0.0;
    st->b2 = 3.0;
    st->b3 = -2.0;
    st->done = 0;
  }
}

// The refined P (in buf[1]) goes to the caller's buffer.
__global__ void refine_copy_kernel(const BatchMat* __restrict__ mats) {
  const BatchMat& M = mats[blockIdx.y];
  if (M.state->done) return;
  const int64_t n = M.n;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n * n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    M.buf[0][i * M.ldp + j] = M.buf[1][e];
  }
}

// tr(P' H) of each refined matrix from the grouped measures' partial sums
// (diagonal and upper P H, the same fixed order as the stopping rules'), and
// the matrix done again.
__global__ void refine_end_kernel(const BatchMat* __restrict__ mats, int nmats, const double* __restrict__ part) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nmats; b += gridDim.x * blockDim.x) {
    PurifyState* st = mats[b].state;
    if (st->done) continue;
    double d = 0.0, u = 0.0;
    for (int k = 0; k < kMeasBlk; ++k) {
      d += part[(static_cast<int64_t>(b) * kMeasBlk + k) * 8 + 6];
      u += part[(static_cast<int64_t>(b) * kMeasBlk + k) * 8 + 7];
    }
    st->energy_refined = d + 2.0 * u;
    st->done = 1;
  }
}

// ---------------------------------------------------------------- host side
struct BatchLayout {
  size_t mats, tiles, row_start, partials, err, counter, active, scratch, tune_ws, total;
  std::vector<size_t> state, rowbuf, expsP, expsX, buf1, X2, planesP, planesX;
  std::vector<int64_t> n_pad, k_pad;
  int ntiles;
  size_t tune_bytes;
};

struct Carve {
  size_t cur = 0;
  size_t take(size_t bytes, size_t align = 256) {
    cur = (cur + align - 1) / align * align;
    const size_t o = cur;
    cur += bytes;
    return o;
  }
};

int tiles_of(int64_t n_pad, int bn) {
  const int tm = static_cast<int>(n_pad / 128), tn = static_cast<int>(n_pad / bn);
  int cnt = 0;
  for (int bj = 0; bj < tn; ++bj) cnt += std::min(tm, bn * (bj + 1) / 128);
  return cnt;
}

BatchLayout batch_layout(int batch, const int64_t* n, int s_max, int beta) {
  BatchLayout L;
  Carve c;
  const int eb = beta == 5 ? 1 : 2;  // E4M3 bytes or bf16 planes (tcgen05 executor)
  const int64_t kq = beta == 5 ? kPadK8 : kPadK;
  L.mats = c.take(sizeof(BatchMat) * batch, 128);
  L.ntiles = 0;
  for (int b = 0; b < batch; ++b) L.ntiles += tiles_of(round_up(n[b], 256), 128);  // the larger of the two counts
  L.tiles = c.take(sizeof(int4) * std::max(L.ntiles, 1));
  L.row_start = c.take(sizeof(int64_t) * (batch + 1));
  L.partials = c.take(sizeof(double) * 8 * kMeasBlk * batch);
  L.err = c.take(sizeof(int));
  L.counter = c.take(sizeof(int));
  L.active = c.take(sizeof(int));
  L.scratch = c.take(tc_scratch_bytes());
  int64_t nmax = 2;
  for (int b = 0; b < batch; ++b) {
    const int64_t np = round_up(n[b], 256), kp = round_up(n[b], kq);
    L.n_pad.push_back(np);
    L.k_pad.push_back(kp);
    L.state.push_back(c.take(sizeof(PurifyState)));
    L.rowbuf.push_back(c.take(gershgorin_rowbuf_bytes(n[b])));
    L.expsP.push_back(c.take(sizeof(int32_t) * np));
    L.expsX.push_back(c.take(sizeof(int32_t) * np));
    L.buf1.push_back(c.take(sizeof(double) * n[b] * n[b]));
    L.X2.push_back(c.take(sizeof(double) * n[b] * n[b]));
    L.planesP.push_back(c.take(static_cast<size_t>(s_max) * np * kp * eb));
    L.planesX.push_back(c.take(static_cast<size_t>(s_max) * np * kp * eb));
    nmax = std::max(nmax, n[b]);
  }
  // room for the slice-count tuner's single-matrix runs on the largest matrix
  dmp_opts t{};
  t.mode = beta == 8 ? DMP_OZAKI_BF16 : (beta == 5 ? DMP_OZAKI_E4M3 : DMP_OZAKI_INT8);
  t.slices = max_slices(t.mode);
  t.executor = DMP_EXEC_TC;
  size_t tb = 0;
  dmp_workspace_size(nmax, &t, &tb);
  L.tune_bytes = tb;
  L.tune_ws = c.take(tb);
  L.total = c.cur;
  return L;
}

struct TuneKey {
  std::vector<int64_t> n;
  int mode;
  bool operator<(const TuneKey& o) const { return std::tie(mode, n) < std::tie(o.mode, o.n); }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tuned;  // -> (slices, tile shape cfg)
std::atomic<int> g_forced_tile{0};                // dmp_set_batched_tile: 0 = tuner

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_graph_mu;
std::map<std::string, GraphEntry> g_graphs;

cudaStream_t capture_stream() {
  static cudaStream_t s = nullptr;
  if (s == nullptr) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  return s;
}

bool make_map(CUtensorMap* tm, const void* planes, int64_t k_pad, int64_t rows_total, int box_rows, bool f8) {
  return make_plane_map_ext(tm, planes, k_pad, rows_total, box_rows, f8);
}

bool batch_mode(int32_t mode) { return mode == DMP_OZAKI_INT8 || mode == DMP_OZAKI_BF16 || mode == DMP_OZAKI_E4M3; }

#define DMP_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return DMP_ERR_CUDA; \
  } while (0)

inline char* at(void* base, size_t off) { return static_cast<char*>(base) + off; }

}  // namespace
}  // namespace dmp

using namespace dmp;

extern "C" {

int dmp_batched_workspace_size(int32_t batch, const int64_t* n, const dmp_opts* opts, size_t* bytes) {
  if (batch <= 0 || n == nullptr || opts == nullptr || bytes == nullptr) return DMP_ERR_INVALID_ARG;
  for (int b = 0; b < batch; ++b)
    if (n[b] < 2) return DMP_ERR_INVALID_ARG;
  if (!batch_mode(opts->mode)) return DMP_ERR_UNSUPPORTED;
  const int beta = beta_of(opts->mode);
  const int s_max =
      std::max(opts->slices > 0 ? opts->slices : max_slices(opts->mode), std::max(opts->refine_slices, 0));
  *bytes = batch_layout(batch, n, s_max, beta).total;
  return DMP_OK;
}

int dm_purify_batched(int32_t batch, const double* const* H, const int64_t* n, const int64_t* n_occ,
                      double* const* P, const dmp_opts* opts, dmp_info* infos, void* ws, size_t ws_bytes,
                      void* stream) {
  if (batch <= 0 || H == nullptr || n == nullptr || n_occ == nullptr || P == nullptr || opts == nullptr ||
      ws == nullptr)
    return DMP_ERR_INVALID_ARG;
  if (!batch_mode(opts->mode)) return DMP_ERR_UNSUPPORTED;
  if (opts->executor != DMP_EXEC_AUTO && opts->executor != DMP_EXEC_TC) return DMP_ERR_UNSUPPORTED;
  if (opts->refine_slices < 0) return DMP_ERR_UNSUPPORTED;  // the refinement step runs Ozaki products only
  if (opts->flags & DMP_FLAG_FP32_STORAGE) return DMP_ERR_UNSUPPORTED;
  if (opts->late_slices != 0) return DMP_ERR_UNSUPPORTED;  // one slice count per batched launch
  if (opts->method != DMP_METHOD_PM) return DMP_ERR_UNSUPPORTED;  // canonical purification only
  const int beta = beta_of(opts->mode);
  const int smax_mode = max_slices(opts->mode);
  const bool f8 = beta == 5;
  if (opts->slices < 0 || opts->slices > smax_mode) return DMP_ERR_INVALID_ARG;
  const int refine = opts->refine_slices;  // 0: none
  if (refine > smax_mode) return DMP_ERR_INVALID_ARG;
  for (int b = 0; b < batch; ++b) {
    if (H[b] == nullptr || P[b] == nullptr || n[b] < 2 || n_occ[b] <= 0 || n_occ[b] >= n[b])
      return DMP_ERR_INVALID_ARG;
    // exact int32 level sums: s k dmax^2 < 2^31 (dmax 127, 128 or 16)
    const double dmax = digit_max(opts->mode);
    if (static_cast<double>(smax_mode) * n[b] * dmax * dmax >= 2147483648.0) return DMP_ERR_UNSUPPORTED;
  }
  const int s_cap = std::max(opts->slices > 0 ? opts->slices : smax_mode, refine);
  const BatchLayout L = batch_layout(batch, n, s_cap, beta);
  if (ws_bytes < L.total) return DMP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int max_iter = opts->max_iter == 0 ? 100 : opts->max_iter;
  const double tol = opts->tol == 0.0 ? 1e-10 : opts->tol;

  BatchMat* dmats = reinterpret_cast<BatchMat*>(at(ws, L.mats));
  int4* dtiles = reinterpret_cast<int4*>(at(ws, L.tiles));
  int64_t* drow = reinterpret_cast<int64_t*>(at(ws, L.row_start));
  double* dpart = reinterpret_cast<double*>(at(ws, L.partials));
  int* derr = reinterpret_cast<int*>(at(ws, L.err));
  int* dcounter = reinterpret_cast<int*>(at(ws, L.counter));
  double* scratch = reinterpret_cast<double*>(at(ws, L.scratch));
  const int64_t nmax_idx = std::max_element(n, n + batch) - n;

  // ---- autotune: slice count (accuracy) and tile width (speed), cached per shape
  TuneKey key{std::vector<int64_t>(n, n + batch),
              opts->mode * 16 + opts->slices + (tc_pairs_available() ? 1024 : 0) + 2048 * refine};
  int s = opts->slices, cfg = 256;
  bool tuned = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      s = it->second.first;
      cfg = it->second.second;
      tuned = true;
    }
  }
  // a cached entry made while the tile shape was forced holds the slice count only
  const bool tile_tuned = tuned && cfg != 0;
  if (cfg == 0) cfg = 256;
  if (!tuned && s == 0) {
    const double target = opts->energy_tol > 0.0 ? opts->energy_tol : 1e-8;
    const int64_t nb = n[nmax_idx];
    double* Pt = reinterpret_cast<double*>(at(ws, L.buf1[nmax_idx]));
    std::vector<double> E(static_cast<size_t>(smax_mode) + 2, 0.0);
    auto energy_at = [&](int sc, double* out) -> int {
      dmp_opts t{};
      t.mode = opts->mode;
      t.slices = sc;
      t.refine_slices = refine;  // compared after the refinement step when the call has one
      t.executor = DMP_EXEC_TC;
      t.max_iter = max_iter;
      t.tol = tol;
      dmp_info inf;
      const int r = dm_purify(H[nmax_idx], nb, nb, n_occ[nmax_idx], &t, Pt, nb, &inf, at(ws, L.tune_ws),
                              L.tune_bytes, nullptr, 0, st);
      if (r < 0) return r;
      *out = inf.energy;
      return DMP_OK;
    };
    s = smax_mode;
    for (int sc = 4; sc + 2 <= smax_mode; ++sc) {
      double e0 = 0.0, e2 = 0.0;
      int r = energy_at(sc, &e0);
      if (r < 0) return r;
      r = energy_at(sc + 2, &e2);
      if (r < 0) return r;
      if (std::fabs(e0 - e2) <= target * std::fabs(e2)) {
        s = sc;
        break;
      }
    }
  } else if (!tuned && s > 0) {
    // keep the caller's s
  }
  if (s > s_cap) return DMP_ERR_WORKSPACE;
  const int forced = g_forced_tile.load();
  if (forced != 0) {
    if ((forced == 128 && f8) || (forced == 512 && !tc_pairs_available())) return DMP_ERR_UNSUPPORTED;
    cfg = forced;
  }

  // ---- descriptors
  std::vector<BatchMat> hm(batch);
  std::vector<int64_t> hrow(batch + 1, 0);
  for (int b = 0; b < batch; ++b) {
    BatchMat& M = hm[b];
    std::memset(&M, 0, sizeof(M));
    M.n = n[b];
    M.n_occ = n_occ[b];
    M.ldh = n[b];
    M.ldp = n[b];
    M.n_pad = L.n_pad[b];
    M.k_pad = L.k_pad[b];
    M.s = s;
    M.buf[0] = P[b];
    M.buf[1] = reinterpret_cast<double*>(at(ws, L.buf1[b]));
    M.X2 = reinterpret_cast<double*>(at(ws, L.X2[b]));
    M.H = H[b];
    M.planesP = at(ws, L.planesP[b]);
    M.planesX = at(ws, L.planesX[b]);
    M.expsP = reinterpret_cast<int32_t*>(at(ws, L.expsP[b]));
    M.expsX = reinterpret_cast<int32_t*>(at(ws, L.expsX[b]));
    M.state = reinterpret_cast<PurifyState*>(at(ws, L.state[b]));
    hrow[b + 1] = hrow[b] + M.n_pad;
  }
  // tile shapes of the grouped product: cfg 128 and 256 are single CTAs on
  // 128 x cfg tiles, cfg 512 is CTA pairs on 256 x 256 tiles (each CTA stages
  // 128 rows of A and 128 of the 256 B rows)
  auto cfg_bn = [](int cfg) { return cfg == 128 ? 128 : 256; };
  auto cfg_pair = [](int cfg) { return cfg == 512; };
  auto build_maps = [&](int cfg) -> bool {
    const int box_b = cfg_pair(cfg) ? cfg_bn(cfg) / 2 : cfg_bn(cfg);
    for (int b = 0; b < batch; ++b) {
      BatchMat& M = hm[b];
      const int64_t rows = static_cast<int64_t>(M.s) * M.n_pad;
      if (!make_map(&M.tmPa, M.planesP, M.k_pad, rows, 128, f8)) return false;
      if (!make_map(&M.tmPb, M.planesP, M.k_pad, rows, box_b, f8)) return false;
      if (!make_map(&M.tmXb, M.planesX, M.k_pad, rows, box_b, f8)) return false;
    }
    return true;
  };
  // matrices by decreasing size: their tiles are listed largest first, so the
  // CTAs that take tiles from the counter finish at about the same time
  std::vector<int> by_size(batch);
  for (int b = 0; b < batch; ++b) by_size[b] = b;
  std::stable_sort(by_size.begin(), by_size.end(), [&](int x, int y) { return n[x] > n[y]; });
  auto build_tiles = [&](int cfg, std::vector<int4>& out) {
    out.clear();
    const int tile_n = cfg_bn(cfg), bm = cfg_pair(cfg) ? 256 : 128;
    // column blocks outermost within each matrix, so CTAs running together
    // work on the same matrix and share its B blocks; only tiles holding some
    // element with row <= column
    for (int b : by_size) {
      const int tm = static_cast<int>(hm[b].n_pad / bm), tn = static_cast<int>(hm[b].n_pad / tile_n);
      for (int bj = 0; bj < tn; ++bj)
        for (int bi = 0; bi < std::min(tm, tile_n * (bj + 1) / bm); ++bi) out.push_back(make_int4(b, bi, bj, 0));
    }
  };
  auto init_states = [&]() -> int {
    for (int b = 0; b < batch; ++b) {
      PurifyState init;
      std::memset(&init, 0, sizeof(init));
      init.tol = tol;
      init.energy_tol = opts->energy_tol;
      init.max_iter = max_iter;
      init.status = DMP_NOT_CONVERGED;
      DMP_CUDA(cudaMemcpyAsync(hm[b].state, &init, sizeof(init), cudaMemcpyHostToDevice, st));
      DMP_CUDA(launch_gershgorin_init(H[b], n[b], n[b], n_occ[b], reinterpret_cast<double*>(at(ws, L.rowbuf[b])),
                                      hm[b].state, P[b], n[b], st));
    }
    DMP_CUDA(cudaStreamSynchronize(st));  // keeps the host copies alive until used
    return DMP_OK;
  };
  const int tbeta = beta;
  std::vector<int4> htiles;
  DMP_CUDA(cudaMemcpyAsync(drow, hrow.data(), sizeof(int64_t) * (batch + 1), cudaMemcpyHostToDevice, st));

  if (!tile_tuned && forced == 0) {
    // tile shape: time the P^2 product of the batch's initial guesses with each
    // (128 x 128 and 128 x 256 single CTAs, 256 x 256 CTA pairs; E4M3 digits run
    // on 256-column tiles only)
    float best = 1e30f;
    int best_cfg = 256;
    int rc = init_states();
    if (rc != DMP_OK) return rc;
    std::vector<int> cands = f8 ? std::vector<int>{256} : std::vector<int>{128, 256};
    if (tc_pairs_available()) cands.push_back(512);
    for (int cand : cands) {
      if (!build_maps(cand)) return DMP_ERR_CUDA;
      build_tiles(cand, htiles);
      DMP_CUDA(cudaMemcpyAsync(dmats, hm.data(), sizeof(BatchMat) * batch, cudaMemcpyHostToDevice, st));
      DMP_CUDA(cudaMemcpyAsync(dtiles, htiles.data(), sizeof(int4) * htiles.size(), cudaMemcpyHostToDevice, st));
      DMP_CUDA(launch_split_grouped(dmats, drow, batch, hrow[batch], 0, tbeta, s, st));
      cudaEvent_t e0, e1;
      DMP_CUDA(cudaEventCreate(&e0));
      DMP_CUDA(cudaEventCreate(&e1));
      DMP_CUDA(cudaEventRecord(e0, st));
      DMP_CUDA(launch_ozaki_tc_grouped(dmats, dtiles, static_cast<int>(htiles.size()), cfg_bn(cand), cfg_pair(cand),
                                       tbeta, 0, 0, derr, scratch, dcounter, st));
      DMP_CUDA(cudaEventRecord(e1, st));
      DMP_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      DMP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms < best) {
        best = ms;
        best_cfg = cand;
      }
    }
    cfg = best_cfg;
  }
  if (!tuned || (!tile_tuned && forced == 0)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = std::make_pair(s, forced != 0 ? 0 : cfg);  // 0: tile shape not tuned yet
  }

  // ---- the real run
  if (!build_maps(cfg)) return DMP_ERR_CUDA;
  build_tiles(cfg, htiles);
  DMP_CUDA(cudaMemcpyAsync(dmats, hm.data(), sizeof(BatchMat) * batch, cudaMemcpyHostToDevice, st));
  DMP_CUDA(cudaMemcpyAsync(dtiles, htiles.data(), sizeof(int4) * htiles.size(), cudaMemcpyHostToDevice, st));
  DMP_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), st));
  {
    const int rc = init_states();
    if (rc != DMP_OK) return rc;
  }
  const int ntiles = static_cast<int>(htiles.size());

  const bool stream_mode = (opts->flags & DMP_FLAG_BATCHED_STREAM) != 0;
  // graph: WHILE(any matrix running) { two iterations }, cached per argument set
  std::string gkey(reinterpret_cast<const char*>(hm.data()), sizeof(BatchMat) * batch);
  gkey.append(reinterpret_cast<const char*>(&ws), sizeof(ws));
  gkey.append(reinterpret_cast<const char*>(&cfg), sizeof(cfg));
  gkey.append(reinterpret_cast<const char*>(&tbeta), sizeof(tbeta));  // the digit rule picks the kernels
  cudaGraphExec_t exec = nullptr;
  if (!stream_mode) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto it = g_graphs.find(gkey);
    if (it != g_graphs.end()) exec = it->second.exec;
  }
  if (!stream_mode && exec == nullptr) {
    GraphEntry ge;
    DMP_CUDA(cudaGraphCreate(&ge.graph, 0));
    cudaGraphConditionalHandle cond;
    DMP_CUDA(cudaGraphConditionalHandleCreate(&cond, ge.graph, 1, cudaGraphCondAssignDefault));
    // cudaGraphNodeParams has no default constructor in C++: zeroed raw storage
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    DMP_CUDA(cudaGraphAddNode(&node, ge.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = capture_stream();
    DMP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    for (int cur = 0; cur < 2; ++cur) {
      launch_split_grouped(dmats, drow, batch, hrow[batch], cur, tbeta, s, cs);
      launch_ozaki_tc_grouped(dmats, dtiles, ntiles, cfg_bn(cfg), cfg_pair(cfg), tbeta, 0, cur, derr, scratch,
                              dcounter, cs);
      launch_measure_grouped(dmats, batch, cur, dpart, cond, 1, nullptr, cs);
      launch_split_grouped(dmats, drow, batch, hrow[batch], 2, tbeta, s, cs);
      launch_ozaki_tc_grouped(dmats, dtiles, ntiles, cfg_bn(cfg), cfg_pair(cfg), tbeta, 1, cur, derr, scratch,
                              dcounter, cs);
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    if (ce != cudaSuccess) return DMP_ERR_CUDA;
    DMP_CUDA(cudaGraphInstantiate(&ge.exec, ge.graph, 0));
    exec = ge.exec;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graphs[gkey] = ge;
  }
  if (stream_mode) {
    // the graph body as plain launches; the host reads the stopping rules'
    // verdict after every two iterations (the graph's condition check)
    int* dactive = reinterpret_cast<int*>(at(ws, L.active));
    for (int it = 0; it < max_iter; it += 2) {
      for (int cur = 0; cur < 2; ++cur) {
        DMP_CUDA(launch_split_grouped(dmats, drow, batch, hrow[batch], cur, tbeta, s, st));
        DMP_CUDA(launch_ozaki_tc_grouped(dmats, dtiles, ntiles, cfg_bn(cfg), cfg_pair(cfg), tbeta, 0, cur, derr,
                                         scratch, dcounter, st));
        DMP_CUDA(launch_measure_grouped(dmats, batch, cur, dpart, cudaGraphConditionalHandle{}, 0, dactive, st));
        DMP_CUDA(launch_split_grouped(dmats, drow, batch, hrow[batch], 2, tbeta, s, st));
        DMP_CUDA(launch_ozaki_tc_grouped(dmats, dtiles, ntiles, cfg_bn(cfg), cfg_pair(cfg), tbeta, 1, cur, derr,
                                         scratch, dcounter, st));
      }
      int active = 0;
      DMP_CUDA(cudaMemcpyAsync(&active, dactive, sizeof(int), cudaMemcpyDeviceToHost, st));
      DMP_CUDA(cudaStreamSynchronize(st));
      if (!active) break;
    }
  } else {
    DMP_CUDA(cudaGraphLaunch(exec, st));
    count_launch();
  }
  DMP_CUDA(launch_finish_grouped(dmats, batch, st));  // every iterate in the caller's P

  if (refine > 0) {
    // ---- refinement step: X^2 = P P and P' = 3 X^2 - 2 P X^2 with r-slice
    // products over the same tiles, for every matrix that ended without an
    // error (the others stay done and are skipped), then tr(P' H)
    for (int b = 0; b < batch; ++b) hm[b].s = refine;
    if (!build_maps(cfg)) return DMP_ERR_CUDA;
    DMP_CUDA(cudaMemcpyAsync(dmats, hm.data(), sizeof(BatchMat) * batch, cudaMemcpyHostToDevice, st));
    {
      ProfScope prof(DMP_PROF_OTHER, st);
      refine_begin_kernel<<<1, 256, 0, st>>>(dmats, batch);
      count_launch();
      DMP_CUDA(cudaGetLastError());
    }
    DMP_CUDA(launch_split_grouped(dmats, drow, batch, hrow[batch], 0, tbeta, refine, st));
    DMP_CUDA(launch_ozaki_tc_grouped(dmats, dtiles, ntiles, cfg_bn(cfg), cfg_pair(cfg), tbeta, 0, 0, derr, scratch,
                                     dcounter, st));
    DMP_CUDA(launch_split_grouped(dmats, drow, batch, hrow[batch], 2, tbeta, refine, st));
    DMP_CUDA(launch_ozaki_tc_grouped(dmats, dtiles, ntiles, cfg_bn(cfg), cfg_pair(cfg), tbeta, 1, 0, derr, scratch,
                                     dcounter, st));
    {
      // the grouped measures' partial sums of P' (buf[1]) give its P H sums
      // (no stopping rules: those would take P' for another iterate)
      ProfScope prof(DMP_PROF_MEASURE, st);
      measure_grouped_kernel<<<dim3(kMeasBlk, batch), 256, 0, st>>>(dmats, 1, dpart);
      count_launch();
      DMP_CUDA(cudaGetLastError());
    }
    {
      ProfScope prof(DMP_PROF_OTHER, st);
      refine_copy_kernel<<<dim3(64, batch), 256, 0, st>>>(dmats);
      refine_end_kernel<<<1, 256, 0, st>>>(dmats, batch, dpart);
      count_launch(2);
      DMP_CUDA(cudaGetLastError());
    }
  }

  std::vector<PurifyState> fin(batch);
  for (int b = 0; b < batch; ++b)
    DMP_CUDA(cudaMemcpyAsync(&fin[b], hm[b].state, sizeof(PurifyState), cudaMemcpyDeviceToHost, st));
  int flag = 0;
  DMP_CUDA(cudaMemcpyAsync(&flag, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  if (flag) return DMP_ERR_TIMEOUT;
  int worst = DMP_OK;
  for (int b = 0; b < batch; ++b) {
    const PurifyState& f = fin[b];
    if (infos != nullptr) {
      dmp_info& I = infos[b];
      I.status = f.status;
      I.iters = f.iter;
      const bool refined = refine > 0 && f.status >= 0;
      I.slices_used = s;
      I.executor_used = DMP_EXEC_TC;
      I.energy = refined ? f.energy_refined : f.energy;
      I.band_energy = 2.0 * I.energy;
      I.idem = std::sqrt(f.idem2);
      I.trace = f.t1;
      I.c_last = f.c;
      I.h_min = f.h_min;
      I.h_max = f.h_max;
      I.energy_unrefined = f.energy;
      I.refined = refined ? 1 : 0;
    }
    worst = std::max(worst, f.status);
  }
  for (int b = 0; b < batch; ++b)
    if (fin[b].status < 0) return fin[b].status;  // the first member error (every report is filled)
  return worst;
}

}  // extern "C"

namespace dmp {

cudaError_t launch_measure_grouped(const BatchMat* mats, int nmats, int cur, double* partials,
                                   cudaGraphConditionalHandle cond, int set_cond, int* active,
                                   cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  measure_grouped_kernel<<<dim3(kMeasBlk, nmats), 256, 0, st>>>(mats, cur, partials);
  measure_grouped_final_kernel<<<1, 256, 0, st>>>(mats, nmats, partials, cond, set_cond, active);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_finish_grouped(const BatchMat* mats, int nmats, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  finish_grouped_kernel<<<dim3(64, nmats), 256, 0, st>>>(mats);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dmp

extern "C" int dmp_set_batched_tile(int tile) {
  if (tile != 0 && tile != 128 && tile != 256 && tile != 512) return DMP_ERR_INVALID_ARG;
  return dmp::g_forced_tile.exchange(tile);
}
