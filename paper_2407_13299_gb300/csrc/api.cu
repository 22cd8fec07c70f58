// C-ABI entry points of libdmp (declared in include/dmp.h).
//
// Host orchestration only: argument checks, workspace carving and kernel
// launches. Every arithmetic step of the path runs in the kernels of this
// library.

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dmp_internal.cuh"

namespace dmp {

std::atomic<long long> g_launches{0};

namespace {

constexpr size_t kAlign = 256;

// Sequential carving of a workspace into aligned regions.
struct Carver {
  size_t cur = 0;
  size_t take(size_t bytes) {
    const size_t off = cur;
    cur = (cur + bytes + kAlign - 1) / kAlign * kAlign;
    return off;
  }
};

struct Opts {
  int mode, s, beta, executor, max_iter, every;
  double tol, energy_tol;
  int refine;  // 0 off, -1 FP64 products, > 0 Ozaki slices of the refinement step
  int method;  // DMP_METHOD_*
  bool store32;  // DMP_FLAG_FP32_STORAGE
  int late_s;    // late-slice schedule: 0 off, else the slice count after the switch
  double late_idem;
};

int normalize(const dmp_opts* o, Opts& out) {
  if (o == nullptr) return DMP_ERR_INVALID_ARG;
  out.mode = o->mode;
  if (out.mode != DMP_FP64 && out.mode != DMP_OZAKI_INT8 && out.mode != DMP_OZAKI_BF16 &&
      out.mode != DMP_OZAKI_E4M3)
    return DMP_ERR_INVALID_ARG;
  out.beta = beta_of(out.mode);
  out.s = o->slices == 0 ? 7 : o->slices;
  const int smax = max_slices(out.mode);
  if (out.mode != DMP_FP64) {
    if (out.s < 1 || out.s > smax) return DMP_ERR_INVALID_ARG;
  } else {
    out.s = 0;
  }
  out.executor = o->executor;
  if (out.executor < DMP_EXEC_AUTO || out.executor > DMP_EXEC_TC) return DMP_ERR_INVALID_ARG;
  // the tcgen05 executor is the fast one on this GPU (bf16 tensor rate >> int8 mma.sync rate)
  if (out.mode != DMP_FP64 && out.executor == DMP_EXEC_AUTO) out.executor = DMP_EXEC_TC;
  if ((out.mode == DMP_OZAKI_BF16 || out.mode == DMP_OZAKI_E4M3) && out.executor == DMP_EXEC_IMMA)
    return DMP_ERR_UNSUPPORTED;
  if (out.mode == DMP_FP64) out.executor = 0;
  out.max_iter = o->max_iter == 0 ? 100 : o->max_iter;
  if (out.max_iter < 0) return DMP_ERR_INVALID_ARG;
  out.every = o->checkpoint_every == 0 ? 8 : o->checkpoint_every;
  if (out.every < 1) return DMP_ERR_INVALID_ARG;
  out.tol = o->tol == 0.0 ? 1e-10 : o->tol;
  out.energy_tol = o->energy_tol;
  if (!(out.tol >= 0.0) || !(out.energy_tol >= 0.0)) return DMP_ERR_INVALID_ARG;
  out.store32 = (o->flags & DMP_FLAG_FP32_STORAGE) != 0;
  out.method = o->method;
  if (out.method < DMP_METHOD_PM || out.method > DMP_METHOD_SP2) return DMP_ERR_INVALID_ARG;
  out.refine = o->refine_slices;
  if (out.refine != 0 && out.mode == DMP_FP64) out.refine = -1;
  if (out.refine < -1 || out.refine > smax) return DMP_ERR_INVALID_ARG;
  out.late_s = out.mode == DMP_FP64 ? 0 : o->late_slices;
  out.late_idem = o->late_idem;
  if (out.late_s < 0 || out.late_s > smax || !(out.late_idem >= 0.0)) return DMP_ERR_INVALID_ARG;
  if (out.late_s > 0 && out.method != DMP_METHOD_PM) return DMP_ERR_UNSUPPORTED;
  return DMP_OK;
}

// Level sums stay exact in int32 while s k dmax^2 < 2^31 (both executors keep
// them in int32).
bool levels_fit_int32(int64_t k, int s, int mode) {
  const double dmax = digit_max(mode);
  const double bound = static_cast<double>(s) * static_cast<double>(k) * dmax * dmax;
  return bound < 2147483648.0;
}

// digit plane element: int8 (IMMA), bfloat16 (tcgen05) or E4M3 bytes (E4M3 mode)
int elem_bytes(const Opts& o) { return (o.executor == DMP_EXEC_TC && o.mode != DMP_OZAKI_E4M3) ? 2 : 1; }
int elem_kind(const Opts& o) {
  if (o.mode == DMP_OZAKI_E4M3) return 4;
  return o.executor == DMP_EXEC_TC ? 3 : 1;
}
// K padding of the digit planes: two swizzle atoms of the paired tcgen05 kernel
int64_t k_pad_of(const Opts& o, int64_t k) {
  return round_up(std::max<int64_t>(k, 1), o.mode == DMP_OZAKI_E4M3 ? kPadK8 : kPadK);
}
// digit-plane rows are padded to the executor's tile height (tcgen05: 256 so
// that one plane set serves as A (128-row tiles) and B (256-row tiles))
int64_t row_pad(int executor) { return executor == DMP_EXEC_TC ? 256 : kTileM; }

#define DMP_CUDA(call)                       \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return DMP_ERR_CUDA; \
  } while (0)

// ---------------------------------------------------------------- dm_purify layout
struct PurifyLayout {
  size_t state, partials, rowbuf, expsP, expsX, err, Palt, X2, planesP, planesX, scratch, split, total;
  int64_t n_pad, k_pad;
};

PurifyLayout purify_layout(int64_t n, const Opts& o) {
  PurifyLayout L;
  Carver c;
  L.n_pad = round_up(n, o.mode == DMP_FP64 ? kTileM : row_pad(o.executor));
  L.k_pad = k_pad_of(o, n);
  L.state = c.take(sizeof(PurifyState));
  L.partials = c.take(static_cast<size_t>(kMeasureBlocks) * 10 * sizeof(double));  // 8 measures, 10 for SP2 / TRS4
  L.rowbuf = c.take(gershgorin_rowbuf_bytes(n));
  L.expsP = c.take(static_cast<size_t>(L.n_pad) * sizeof(int32_t));
  L.expsX = c.take(static_cast<size_t>(L.n_pad) * sizeof(int32_t));
  L.err = c.take(sizeof(int32_t));
  L.Palt = c.take(static_cast<size_t>(n) * n * sizeof(double));
  L.X2 = c.take(static_cast<size_t>(n) * n * sizeof(double));
  if (o.mode != DMP_FP64) {
    // room for the refinement step's slices too
    const int smax = std::max(std::max(o.s, o.refine), o.late_s);
    const size_t plane = static_cast<size_t>(smax) * L.n_pad * L.k_pad * elem_bytes(o);
    L.planesP = c.take(plane);
    L.planesX = c.take(plane);
  } else {
    L.planesP = L.planesX = 0;
  }
  L.scratch = (o.mode != DMP_FP64 && o.executor == DMP_EXEC_TC) ? c.take(tc_scratch_bytes()) : 0;
  L.split = (o.mode != DMP_FP64 && o.executor == DMP_EXEC_TC) ? c.take(tc_split_bytes()) : 0;
  L.total = c.cur;
  return L;
}

// One Ozaki product from prepared digit planes on the chosen executor.
// `split_ws` (nullable) is the tcgen05 executor's workspace for split launches (tc_split_bytes).
cudaError_t launch_product(const Opts& o, const void* pa, const void* pb, const int32_t* ea, const int32_t* eb,
                           int64_t m, int64_t n, int64_t rows_a, int64_t rows_b, int64_t k_pad, int sym,
                           const EpiArgs& epi, const int* done, int* err, double* scratch, void* split_ws,
                           cudaStream_t st) {
  if (o.executor == DMP_EXEC_TC)
    return launch_ozaki_tc(pa, pb, ea, eb, m, n, rows_a, rows_b, k_pad, o.s, o.beta, sym, epi, done, err, scratch,
                           split_ws, st);
  return launch_ozaki_imma(static_cast<const int8_t*>(pa), static_cast<const int8_t*>(pb), ea, eb, m, n, rows_a,
                           rows_b, k_pad, o.s, o.beta, sym, epi, done, st);
}

// Tape: header, per-step coefficients, then checkpoints P_0, P_k, P_2k, ...
struct TapeHeader {
  int32_t magic, n, iters, every, n_ckpt, mode, s, executor;
  int32_t status, row_min, row_max, lam_branch;
  double lam, mu, h_min, h_max;
};
constexpr int32_t kTapeMagic = 0x444d5054;  // "DMPT"

struct TapeLayout {
  size_t header, coeffs, ckpt, total;
  int n_ckpt;
};

TapeLayout tape_layout(int64_t n, const Opts& o) {
  TapeLayout T;
  Carver c;
  T.header = c.take(sizeof(TapeHeader));
  T.coeffs = c.take(static_cast<size_t>(o.max_iter + 1) * sizeof(double));
  T.n_ckpt = o.max_iter / o.every + 1;
  T.ckpt = c.take(static_cast<size_t>(T.n_ckpt) * n * n * sizeof(double));
  T.total = c.cur;
  return T;
}

inline char* at(void* base, size_t off) { return static_cast<char*>(base) + off; }

// dm_purify_backward workspace: six n x n matrices (G, G', Y, Z, YP, ZP), the
// recomputed iterates and squares of one checkpoint segment, and the split
// buffers of one product.
struct BackwardLayout {
  size_t state, scalars, p0, partials, err, expsP, expsA, G, Gn, Y, Z, YP, ZP, segP, segX, planesP, planesA,
      scratch, split, total;
  int64_t n_pad, k_pad;
};

BackwardLayout backward_layout(int64_t n, const Opts& o) {
  BackwardLayout B;
  Carver c;
  const size_t nn = static_cast<size_t>(n) * n * sizeof(double);
  B.n_pad = round_up(n, o.mode == DMP_FP64 ? kTileM : row_pad(o.executor));
  B.k_pad = k_pad_of(o, n);
  B.state = c.take(sizeof(PurifyState));
  B.scalars = c.take(sizeof(AdjScalars));
  B.p0 = c.take(sizeof(P0Adjoint));
  B.partials = c.take(304 * 5 * sizeof(double));
  B.err = c.take(sizeof(int32_t));
  B.expsP = c.take(static_cast<size_t>(B.n_pad) * sizeof(int32_t));
  B.expsA = c.take(static_cast<size_t>(B.n_pad) * sizeof(int32_t));
  B.G = c.take(nn);
  B.Gn = c.take(nn);
  B.Y = c.take(nn);
  B.Z = c.take(nn);
  B.YP = c.take(nn);
  B.ZP = c.take(nn);
  B.segP = c.take(nn * o.every);
  B.segX = c.take(nn * o.every);
  if (o.mode != DMP_FP64) {
    const size_t plane = static_cast<size_t>(o.s) * B.n_pad * B.k_pad * elem_bytes(o);
    B.planesP = c.take(plane);
    B.planesA = c.take(plane);
  } else {
    B.planesP = B.planesA = 0;
  }
  B.scratch = (o.mode != DMP_FP64 && o.executor == DMP_EXEC_TC) ? c.take(tc_scratch_bytes()) : 0;
  B.split = (o.mode != DMP_FP64 && o.executor == DMP_EXEC_TC) ? c.take(tc_split_bytes()) : 0;
  B.total = c.cur;
  return B;
}

// Baby steps of the Paterson-Stockmeyer scheme: q = ceil(sqrt(M)); r = ceil(M / q) blocks.
int ps_q(int M) {
  int q = 1;
  while (q * q < M) ++q;
  return q;
}
constexpr int kFoeMaxQ = 128;  // ps_q(DMP_FOE_MAX_TERMS)

// dm_foe workspace: the run state and Gershgorin buffers, the expansion's
// scalars, coefficients, traces and node arrays (sized for the largest M), and
// n x n matrices: for the three-term recurrence H_s, two recurrence terms and
// the product Y; for the Paterson-Stockmeyer scheme the q baby steps T_1 .. T_q
// (H_s = T_1), Y and two Clenshaw (or giant-step) terms. Digit planes of H_s
// (split once), of the current right operand, and of y = T_q (scheme 1).
struct FoeLayout {
  size_t state, rowbuf, scal, coeffs, traces, w, gx, fold, psw, ip, dots, partials, err, Hs, Ta, Tb, Y, Tps, expsH,
      expsT, expsY, planesH, planesT, planesY, scratch, split, total;
  int64_t n_pad, k_pad;
};

FoeLayout foe_layout(int64_t n, const Opts& o, int scheme, int M) {
  FoeLayout F{};
  Carver c;
  const size_t nn = static_cast<size_t>(n) * n * sizeof(double);
  const size_t terms = static_cast<size_t>(2 * kFoeMaxTerms) * sizeof(double);
  F.n_pad = round_up(n, o.mode == DMP_FP64 ? kTileM : row_pad(o.executor));
  F.k_pad = k_pad_of(o, n);
  F.state = c.take(sizeof(PurifyState));
  F.rowbuf = c.take(gershgorin_rowbuf_bytes(n));
  F.scal = c.take(sizeof(FoeScalars));
  F.coeffs = c.take(terms);
  F.traces = c.take(terms);
  F.w = c.take(terms);
  F.gx = c.take(terms);
  F.fold = c.take(terms);
  F.psw = c.take(terms);
  F.ip = c.take(terms);
  F.dots = c.take(static_cast<size_t>(kFoeDotBlocks) * kFoeMaxQ * sizeof(double));
  F.partials = c.take(static_cast<size_t>(kMeasureBlocks) * 10 * sizeof(double));
  F.err = c.take(sizeof(int32_t));
  if (scheme == DMP_FOE_PATERSON_STOCKMEYER) {
    F.Tps = c.take(static_cast<size_t>(ps_q(M)) * nn);
    F.Hs = F.Tps;
  } else {
    F.Hs = c.take(nn);
  }
  F.Ta = c.take(nn);
  F.Tb = c.take(nn);
  F.Y = c.take(nn);
  if (o.mode != DMP_FP64) {
    const size_t plane = static_cast<size_t>(o.s) * F.n_pad * F.k_pad * elem_bytes(o);
    F.expsH = c.take(static_cast<size_t>(F.n_pad) * sizeof(int32_t));
    F.expsT = c.take(static_cast<size_t>(F.n_pad) * sizeof(int32_t));
    F.planesH = c.take(plane);
    F.planesT = c.take(plane);
    if (scheme == DMP_FOE_PATERSON_STOCKMEYER) {
      F.expsY = c.take(static_cast<size_t>(F.n_pad) * sizeof(int32_t));
      F.planesY = c.take(plane);
    }
  }
  F.scratch = (o.mode != DMP_FP64 && o.executor == DMP_EXEC_TC) ? c.take(tc_scratch_bytes()) : 0;
  F.split = (o.mode != DMP_FP64 && o.executor == DMP_EXEC_TC) ? c.take(tc_split_bytes()) : 0;
  F.total = c.cur;
  return F;
}

// Options dm_foe accepts: the product mode, slices and executor only.
int foe_opts(const dmp_opts* opts, Opts& o) {
  const int rc = normalize(opts, o);
  if (rc != DMP_OK) return rc;
  if (o.refine != 0 || o.late_s != 0 || o.method != DMP_METHOD_PM || o.store32) return DMP_ERR_UNSUPPORTED;
  return DMP_OK;
}

}  // namespace
}  // namespace dmp

using namespace dmp;

extern "C" {

const char* dmp_version(void) { return "dmp 0.1 (sm_103a)"; }

long long dmp_launch_count(void) { return g_launches.load(); }

int dmp_set_tc_pairing(int enable) { return set_tc_pairing(enable); }

int dmp_test_stall_next_product(int32_t wait_limit_us) { return set_stall_test(wait_limit_us); }

int dmp_set_tc_split_tiles(int enable) { return set_tc_split_tiles(enable); }

const char* dmp_status_str(int code) {
  switch (code) {
    case DMP_OK: return "DMP_OK";
    case DMP_NOT_CONVERGED: return "DMP_NOT_CONVERGED";
    case DMP_STALLED: return "DMP_STALLED";
    case DMP_C_OUT_OF_RANGE: return "DMP_C_OUT_OF_RANGE";
    case DMP_ERR_INVALID_ARG: return "DMP_ERR_INVALID_ARG";
    case DMP_ERR_NONFINITE: return "DMP_ERR_NONFINITE";
    case DMP_ERR_CUDA: return "DMP_ERR_CUDA";
    case DMP_ERR_TIMEOUT: return "DMP_ERR_TIMEOUT";
    case DMP_ERR_UNSUPPORTED: return "DMP_ERR_UNSUPPORTED";
    case DMP_ERR_WORKSPACE: return "DMP_ERR_WORKSPACE";
    default: return "DMP_UNKNOWN";
  }
}

int dmp_workspace_size(int64_t n, const dmp_opts* opts, size_t* bytes) {
  Opts o;
  const int rc = normalize(opts, o);
  if (rc != DMP_OK) return rc;
  if (n < 2 || bytes == nullptr) return DMP_ERR_INVALID_ARG;
  *bytes = purify_layout(n, o).total;
  return DMP_OK;
}

int dmp_tape_size(int64_t n, const dmp_opts* opts, size_t* bytes) {
  Opts o;
  const int rc = normalize(opts, o);
  if (rc != DMP_OK) return rc;
  if (n < 2 || bytes == nullptr) return DMP_ERR_INVALID_ARG;
  *bytes = tape_layout(n, o).total;
  return DMP_OK;
}

int dm_purify(const double* H, int64_t n, int64_t ldh, int64_t n_occ, const dmp_opts* opts,
              double* P, int64_t ldp, dmp_info* info, void* ws, size_t ws_bytes, void* tape,
              size_t tape_bytes, void* stream) {
  Opts o;
  int rc = normalize(opts, o);
  if (rc != DMP_OK) return rc;
  if (H == nullptr || P == nullptr || ws == nullptr) return DMP_ERR_INVALID_ARG;
  if (n < 2 || ldh < n || ldp < n || n_occ <= 0 || n_occ >= n) return DMP_ERR_INVALID_ARG;
  if (o.mode != DMP_FP64 && !levels_fit_int32(n, o.s, o.mode))
    return DMP_ERR_UNSUPPORTED;
  if (o.refine > 0 && !levels_fit_int32(n, o.refine, o.mode))
    return DMP_ERR_UNSUPPORTED;
  if (o.late_s > 0 && !levels_fit_int32(n, o.late_s, o.mode))
    return DMP_ERR_UNSUPPORTED;
  if ((o.refine != 0 || o.method != DMP_METHOD_PM || o.store32 || o.late_s > 0) && tape != nullptr)
    return DMP_ERR_UNSUPPORTED;
  const PurifyLayout L = purify_layout(n, o);
  if (ws_bytes < L.total) return DMP_ERR_WORKSPACE;
  TapeLayout TL{};
  if (tape != nullptr) {
    TL = tape_layout(n, o);
    if (tape_bytes < TL.total) return DMP_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  PurifyState* state = reinterpret_cast<PurifyState*>(at(ws, L.state));
  double* partials = reinterpret_cast<double*>(at(ws, L.partials));
  double* rowbuf = reinterpret_cast<double*>(at(ws, L.rowbuf));
  int32_t* expsP = reinterpret_cast<int32_t*>(at(ws, L.expsP));
  int32_t* expsX = reinterpret_cast<int32_t*>(at(ws, L.expsX));
  double* Palt = reinterpret_cast<double*>(at(ws, L.Palt));
  double* X2 = reinterpret_cast<double*>(at(ws, L.X2));
  void* planesP = o.mode != DMP_FP64 ? at(ws, L.planesP) : nullptr;
  void* planesX = o.mode != DMP_FP64 ? at(ws, L.planesX) : nullptr;
  int* err = reinterpret_cast<int*>(at(ws, L.err));
  double* scratch = L.scratch ? reinterpret_cast<double*>(at(ws, L.scratch)) : nullptr;
  void* split_ws = L.split ? at(ws, L.split) : nullptr;
  DMP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));

  PurifyState init;
  std::memset(&init, 0, sizeof(init));
  init.tol = o.tol;
  init.energy_tol = o.energy_tol;
  init.max_iter = o.max_iter;
  init.status = DMP_NOT_CONVERGED;
  init.method = o.method;
  init.store32 = o.store32 ? 1 : 0;
  DMP_CUDA(cudaMemcpyAsync(state, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  DMP_CUDA(launch_gershgorin_init(H, n, ldh, n_occ, rowbuf, state, P, ldp, st));

  double* tape_c = tape ? reinterpret_cast<double*>(at(tape, TL.coeffs)) : nullptr;
  double* tape_ck = tape ? reinterpret_cast<double*>(at(tape, TL.ckpt)) : nullptr;

  double* cur = P;
  int64_t ldcur = ldp;
  double* alt = Palt;
  int64_t ldalt = n;
  const int* done = &state->done;
  bool late = false;  // the late-slice schedule has switched
  int late_iters = 0;
  for (int k = 0; k <= o.max_iter; ++k) {
    Opts oi = o;  // this pass's slice count
    if (late) {
      oi.s = o.late_s;
      ++late_iters;
    }
    if (tape != nullptr && k % o.every == 0) {
      DMP_CUDA(cudaMemcpy2DAsync(tape_ck + static_cast<size_t>(k / o.every) * n * n, n * sizeof(double),
                                 cur, ldcur * sizeof(double), n * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, st));
    }
    EpiArgs e2{};
    e2.kind = EPI_SYM_STORE;
    e2.C = X2;
    e2.ldc = n;
    e2.round32 = o.store32 ? 1 : 0;
    if (o.mode == DMP_FP64) {
      DMP_CUDA(launch_gemm_f64(cur, ldcur, cur, ldcur, n, n, n, 1, e2, done, st));
    } else {
      DMP_CUDA(launch_split_rows(cur, n, n, ldcur, oi.s, oi.beta, expsP, planesP, L.n_pad, L.k_pad,
                                 elem_kind(o), nullptr, done, st));
      DMP_CUDA(launch_product(oi, planesP, planesP, expsP, expsP, n, n, L.n_pad, L.n_pad, L.k_pad, 1, e2, done,
                              err, scratch, split_ws, st));
    }
    if (o.method == DMP_METHOD_PM) {
      DMP_CUDA(launch_measure(cur, ldcur, X2, n, H, ldh, n, partials, state, st));
    } else {
      DMP_CUDA(launch_measure_variant(cur, ldcur, X2, n, H, ldh, n, partials, state, st));
    }
    int32_t flags[3] = {0, 0, 0};
    double idem2 = 0.0;
    DMP_CUDA(cudaMemcpyAsync(&flags[0], &state->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DMP_CUDA(cudaMemcpyAsync(&flags[1], err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DMP_CUDA(cudaMemcpyAsync(&flags[2], &state->step_kind, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (o.late_s > 0) DMP_CUDA(cudaMemcpyAsync(&idem2, &state->idem2, sizeof(double), cudaMemcpyDeviceToHost, st));
    DMP_CUDA(cudaStreamSynchronize(st));
    if (flags[1]) return DMP_ERR_TIMEOUT;
    if (flags[0]) break;
    if (o.method != DMP_METHOD_PM) {
      // SP2 / TRS4 step (the weights are on the device)
      if (flags[2] == 0) {
        DMP_CUDA(launch_axpby(cur, ldcur, X2, n, alt, ldalt, n, state, st));
        std::swap(cur, alt);
        std::swap(ldcur, ldalt);
      } else {
        // X' = X2 Z: Z into alt, then the symmetric product written over X
        DMP_CUDA(launch_trs4_z(cur, ldcur, X2, n, alt, ldalt, n, state, st));
        EpiArgs ez{};
        ez.kind = EPI_SYM_STORE;
        ez.C = cur;
        ez.ldc = ldcur;
        ez.round32 = o.store32 ? 1 : 0;
        if (o.mode == DMP_FP64) {
          DMP_CUDA(launch_gemm_f64(X2, n, alt, ldalt, n, n, n, 1, ez, done, st));
        } else {
          DMP_CUDA(launch_split_rows(X2, n, n, n, oi.s, oi.beta, expsX, planesX, L.n_pad, L.k_pad,
                                     elem_kind(o), nullptr, done, st));
          DMP_CUDA(launch_split_rows(alt, n, n, ldalt, oi.s, oi.beta, expsP, planesP, L.n_pad, L.k_pad,
                                     elem_kind(o), nullptr, done, st));
          DMP_CUDA(launch_product(oi, planesX, planesP, expsX, expsP, n, n, L.n_pad, L.n_pad, L.k_pad, 1, ez, done,
                                  err, scratch, split_ws, st));
        }
      }
      continue;
    }
    if (tape != nullptr) {
      DMP_CUDA(cudaMemcpyAsync(tape_c + k, &state->c, sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    EpiArgs e3{};
    e3.kind = EPI_PM_UPDATE;
    e3.C = alt;
    e3.ldc = ldalt;
    e3.P = cur;
    e3.ldp = ldcur;
    e3.X2 = X2;
    e3.ldx = n;
    e3.state = state;
    e3.round32 = o.store32 ? 1 : 0;
    if (o.mode == DMP_FP64) {
      DMP_CUDA(launch_gemm_f64(cur, ldcur, X2, n, n, n, n, 1, e3, done, st));
    } else {
      DMP_CUDA(launch_split_rows(X2, n, n, n, oi.s, oi.beta, expsX, planesX, L.n_pad, L.k_pad,
                                 elem_kind(o), nullptr, done, st));
      DMP_CUDA(launch_product(oi, planesP, planesX, expsP, expsX, n, n, L.n_pad, L.n_pad, L.k_pad, 1, e3, done,
                              err, scratch, split_ws, st));
    }
    std::swap(cur, alt);
    std::swap(ldcur, ldalt);
    // the late-slice schedule switches after an update whose iterate was within late_idem of idempotency
    if (o.late_s > 0 && std::sqrt(idem2) < o.late_idem) late = true;
  }
  // ---- refinement (Sec. "Precision Requirements Sweep"): one McWeeny step in
  // full precision, P' = 3 P^2 - 2 P^3, run as the update with the weights of c = 1/2
  bool refined = false;
  if (o.refine != 0) {
    int32_t status_now = 0;
    DMP_CUDA(cudaMemcpyAsync(&status_now, &state->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DMP_CUDA(cudaStreamSynchronize(st));
    if (status_now >= 0) {
      DMP_CUDA(launch_refine_weights(state, st));
      EpiArgs r2{};
      r2.kind = EPI_SYM_STORE;
      r2.C = X2;
      r2.ldc = n;
      EpiArgs r3{};
      r3.kind = EPI_PM_UPDATE;
      r3.C = alt;
      r3.ldc = ldalt;
      r3.P = cur;
      r3.ldp = ldcur;
      r3.X2 = X2;
      r3.ldx = n;
      r3.state = state;
      if (o.refine < 0) {
        DMP_CUDA(launch_gemm_f64(cur, ldcur, cur, ldcur, n, n, n, 1, r2, nullptr, st));
        DMP_CUDA(launch_gemm_f64(cur, ldcur, X2, n, n, n, n, 1, r3, nullptr, st));
      } else {
        Opts orr = o;
        orr.s = o.refine;
        DMP_CUDA(launch_split_rows(cur, n, n, ldcur, orr.s, orr.beta, expsP, planesP, L.n_pad, L.k_pad,
                                   elem_kind(o), nullptr, nullptr, st));
        DMP_CUDA(launch_product(orr, planesP, planesP, expsP, expsP, n, n, L.n_pad, L.n_pad, L.k_pad, 1, r2, nullptr,
                                err, scratch, split_ws, st));
        DMP_CUDA(launch_split_rows(X2, n, n, n, orr.s, orr.beta, expsX, planesX, L.n_pad, L.k_pad,
                                   elem_kind(o), nullptr, nullptr, st));
        DMP_CUDA(launch_product(orr, planesP, planesX, expsP, expsX, n, n, L.n_pad, L.n_pad, L.k_pad, 1, r3, nullptr,
                                err, scratch, split_ws, st));
      }
      std::swap(cur, alt);
      std::swap(ldcur, ldalt);
      DMP_CUDA(launch_energy(cur, ldcur, H, ldh, n, partials, state, st));
      refined = true;
    }
  }
  if (cur != P) {
    DMP_CUDA(cudaMemcpy2DAsync(P, ldp * sizeof(double), cur, ldcur * sizeof(double), n * sizeof(double), n,
                               cudaMemcpyDeviceToDevice, st));
  }
  PurifyState fin;
  int32_t err_end = 0;
  DMP_CUDA(cudaMemcpyAsync(&fin, state, sizeof(fin), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaMemcpyAsync(&err_end, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  if (err_end) return DMP_ERR_TIMEOUT;
  if (tape != nullptr) {
    TapeHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kTapeMagic;
    h.n = static_cast<int32_t>(n);
    h.iters = fin.iter;
    h.every = o.every;
    h.n_ckpt = TL.n_ckpt;
    h.mode = o.mode;
    h.s = o.s;
    h.executor = o.executor;
    h.status = fin.status;
    h.row_min = fin.row_min;
    h.row_max = fin.row_max;
    h.lam_branch = fin.lam_branch;
    h.lam = fin.lam;
    h.mu = fin.mu;
    h.h_min = fin.h_min;
    h.h_max = fin.h_max;
    DMP_CUDA(cudaMemcpyAsync(at(tape, TL.header), &h, sizeof(h), cudaMemcpyHostToDevice, st));
    DMP_CUDA(cudaStreamSynchronize(st));
  }
  if (info != nullptr) {
    info->status = fin.status;
    info->iters = fin.iter;
    info->slices_used = o.s;
    info->executor_used = o.executor;
    info->energy = refined ? fin.energy_refined : fin.energy;
    info->band_energy = 2.0 * info->energy;
    info->energy_unrefined = fin.energy;
    info->refined = refined ? 1 : 0;
    info->late_iters = late_iters;
    info->idem = std::sqrt(fin.idem2);
    info->trace = fin.t1;
    info->c_last = fin.c;
    info->h_min = fin.h_min;
    info->h_max = fin.h_max;
  }
  return fin.status;
}

// dm_purify_host: device copies of H and P at the front of the workspace,
// dm_purify's own workspace after them.
static size_t host_front_bytes(int64_t n) {
  const size_t nn = static_cast<size_t>(n) * static_cast<size_t>(n) * sizeof(double);
  return 2 * ((nn + 255) / 256 * 256);
}

int dmp_host_workspace_size(int64_t n, const dmp_opts* opts, size_t* bytes) {
  size_t inner = 0;
  const int rc = dmp_workspace_size(n, opts, &inner);
  if (rc != DMP_OK) return rc;
  *bytes = host_front_bytes(n) + inner;
  return DMP_OK;
}

int dm_purify_host(const double* H_host, int64_t n, int64_t ldh, int64_t n_occ, const dmp_opts* opts,
                   double* P_host, int64_t ldp, dmp_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (H_host == nullptr || P_host == nullptr || ws == nullptr || opts == nullptr) return DMP_ERR_INVALID_ARG;
  if (n < 2 || ldh < n || ldp < n) return DMP_ERR_INVALID_ARG;
  size_t need = 0;
  const int rc = dmp_host_workspace_size(n, opts, &need);
  if (rc != DMP_OK) return rc;
  if (ws_bytes < need) return DMP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t front = host_front_bytes(n);
  double* Hd = reinterpret_cast<double*>(ws);
  double* Pd = reinterpret_cast<double*>(static_cast<char*>(ws) + front / 2);
  const size_t row = static_cast<size_t>(n) * sizeof(double);
  // H in: one strided copy on the caller's stream (asynchronous DMA from pinned memory)
  DMP_CUDA(cudaMemcpy2DAsync(Hd, row, H_host, static_cast<size_t>(ldh) * sizeof(double), row, n,
                             cudaMemcpyHostToDevice, st));
  const int status = dm_purify(Hd, n, n, n_occ, opts, Pd, n, info, static_cast<char*>(ws) + front, ws_bytes - front,
                               nullptr, 0, stream);
  if (status < 0) {
    cudaStreamSynchronize(st);  // the copy of H may still read the caller's buffer
    return status;
  }
  // P out, then wait: the caller's host buffer holds P when the call returns
  DMP_CUDA(cudaMemcpy2DAsync(P_host, static_cast<size_t>(ldp) * sizeof(double), Pd, row, row, n,
                             cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  return status;
}

int ozaki_gemm_workspace_size(int64_t m, int64_t n, int64_t k, int32_t mode, int32_t slices,
                              int32_t executor, size_t* bytes) {
  dmp_opts d{};
  d.mode = mode;
  d.slices = slices;
  d.executor = executor;
  Opts o;
  const int rc = normalize(&d, o);
  if (rc != DMP_OK) return rc;
  if (m < 0 || n < 0 || k < 0 || bytes == nullptr) return DMP_ERR_INVALID_ARG;
  if (o.mode == DMP_FP64) {
    *bytes = 0;
    return DMP_OK;
  }
  Carver c;
  const int64_t m_pad = round_up(std::max<int64_t>(m, 1), row_pad(o.executor));
  const int64_t n_pad = round_up(std::max<int64_t>(n, 1), row_pad(o.executor));
  const int64_t k_pad = k_pad_of(o, k);
  c.take(m_pad * sizeof(int32_t));
  c.take(n_pad * sizeof(int32_t));
  c.take(sizeof(int32_t));
  c.take(o.executor == DMP_EXEC_TC ? tc_scratch_bytes() : 0);
  c.take(static_cast<size_t>(o.s) * m_pad * k_pad * elem_bytes(o));
  c.take(static_cast<size_t>(o.s) * n_pad * k_pad * elem_bytes(o));
  c.take(static_cast<size_t>(n) * k * sizeof(double));
  *bytes = c.cur;
  return DMP_OK;
}

static int ozaki_common(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                        int64_t ldb, const EpiArgs& epi, int32_t mode, int32_t slices, int32_t executor,
                        void* ws, size_t ws_bytes, void* stream) {
  dmp_opts d{};
  d.mode = mode;
  d.slices = slices;
  d.executor = executor;
  Opts o;
  const int rc = normalize(&d, o);
  if (rc != DMP_OK) return rc;
  if (m < 0 || n < 0 || k < 0) return DMP_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return DMP_OK;
  if (A == nullptr || B == nullptr || lda < k || ldb < n) return DMP_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.mode == DMP_FP64) {
    if (epi.kind == EPI_LEVELS) return DMP_ERR_INVALID_ARG;
    DMP_CUDA(launch_gemm_f64(A, lda, B, ldb, m, n, k, 0, epi, nullptr, st));
    return DMP_OK;
  }
  if (!levels_fit_int32(k, o.s, o.mode))
    return DMP_ERR_UNSUPPORTED;
  size_t need = 0;
  ozaki_gemm_workspace_size(m, n, k, mode, slices, executor, &need);
  if (ws == nullptr || ws_bytes < need) return DMP_ERR_WORKSPACE;
  Carver c;
  const int64_t m_pad = round_up(m, row_pad(o.executor));
  const int64_t n_pad = round_up(n, row_pad(o.executor));
  const int64_t k_pad = k_pad_of(o, k);
  int32_t* ea = reinterpret_cast<int32_t*>(at(ws, c.take(m_pad * sizeof(int32_t))));
  int32_t* eb = reinterpret_cast<int32_t*>(at(ws, c.take(n_pad * sizeof(int32_t))));
  int* err = reinterpret_cast<int*>(at(ws, c.take(sizeof(int32_t))));
  double* scratch = reinterpret_cast<double*>(at(ws, c.take(o.executor == DMP_EXEC_TC ? tc_scratch_bytes() : 0)));
  void* pa = at(ws, c.take(static_cast<size_t>(o.s) * m_pad * k_pad * elem_bytes(o)));
  void* pb = at(ws, c.take(static_cast<size_t>(o.s) * n_pad * k_pad * elem_bytes(o)));
  double* Bt = reinterpret_cast<double*>(at(ws, c.take(static_cast<size_t>(n) * k * sizeof(double))));
  DMP_CUDA(launch_split_rows(A, m, k, lda, o.s, o.beta, ea, pa, m_pad, k_pad, elem_kind(o), nullptr,
                             nullptr, st));
  DMP_CUDA(launch_transpose(B, k, n, ldb, Bt, st));
  DMP_CUDA(launch_split_rows(Bt, n, k, k, o.s, o.beta, eb, pb, n_pad, k_pad, elem_kind(o), nullptr,
                             nullptr, st));
  if (o.executor == DMP_EXEC_TC) DMP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  DMP_CUDA(launch_product(o, pa, pb, ea, eb, m, n, m_pad, n_pad, k_pad, 0, epi, nullptr, err, scratch, nullptr, st));
  if (o.executor == DMP_EXEC_TC) {
    // report an expired device wait; skipped while the stream is being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DMP_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      int flag = 0;
      DMP_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      DMP_CUDA(cudaStreamSynchronize(st));
      if (flag) return DMP_ERR_TIMEOUT;
    }
  }
  return DMP_OK;
}

int ozaki_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
               int64_t ldb, double* C, int64_t ldc, int32_t mode, int32_t slices, int32_t executor,
               void* ws, size_t ws_bytes, void* stream) {
  if (C == nullptr || ldc < n) return DMP_ERR_INVALID_ARG;
  EpiArgs e{};
  e.kind = EPI_STORE;
  e.C = C;
  e.ldc = ldc;
  return ozaki_common(m, n, k, A, lda, B, ldb, e, mode, slices, executor, ws, ws_bytes, stream);
}

int ozaki_level_sums(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                     int64_t ldb, int32_t* S, int32_t mode, int32_t slices, int32_t executor, void* ws,
                     size_t ws_bytes, void* stream) {
  if (S == nullptr || mode == DMP_FP64) return DMP_ERR_INVALID_ARG;
  EpiArgs e{};
  e.kind = EPI_LEVELS;
  e.levels = S;
  return ozaki_common(m, n, k, A, lda, B, ldb, e, mode, slices, executor, ws, ws_bytes, stream);
}

int ozaki_split(int64_t m, int64_t k, const double* A, int64_t lda, int32_t mode, int32_t slices,
                int32_t executor, int32_t* exps, void* digits, void* ws, size_t ws_bytes, void* stream) {
  dmp_opts d{};
  d.mode = mode;
  d.slices = slices;
  d.executor = executor;
  Opts o;
  const int rc = normalize(&d, o);
  if (rc != DMP_OK) return rc;
  if (o.mode == DMP_FP64) return DMP_ERR_INVALID_ARG;
  if (m <= 0 || k <= 0 || A == nullptr || lda < k || exps == nullptr || digits == nullptr)
    return DMP_ERR_INVALID_ARG;
  size_t need = 0;
  ozaki_gemm_workspace_size(m, 1, k, mode, slices, executor, &need);
  if (ws == nullptr || ws_bytes < need) return DMP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carver c;
  const int64_t m_pad = round_up(m, row_pad(o.executor));
  const int64_t k_pad = k_pad_of(o, k);
  int32_t* ea = reinterpret_cast<int32_t*>(at(ws, c.take(m_pad * sizeof(int32_t))));
  c.take(round_up(1, row_pad(o.executor)) * sizeof(int32_t));
  c.take(sizeof(int32_t));
  const int eb = elem_bytes(o);
  char* pa = at(ws, c.take(static_cast<size_t>(o.s) * m_pad * k_pad * eb));
  DMP_CUDA(launch_split_rows(A, m, k, lda, o.s, o.beta, ea, pa, m_pad, k_pad, elem_kind(o), nullptr,
                             nullptr, st));
  DMP_CUDA(cudaMemcpyAsync(exps, ea, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  for (int i = 0; i < o.s; ++i) {
    DMP_CUDA(cudaMemcpy2DAsync(static_cast<char*>(digits) + static_cast<size_t>(i) * m * k * eb, k * eb,
                               pa + static_cast<size_t>(i) * m_pad * k_pad * eb, k_pad * eb, k * eb, m,
                               cudaMemcpyDeviceToDevice, st));
  }
  return DMP_OK;
}

int dmp_backward_workspace_size(int64_t n, const dmp_opts* opts, size_t* bytes) {
  Opts o;
  const int rc = normalize(opts, o);
  if (rc != DMP_OK) return rc;
  if (n < 2 || bytes == nullptr) return DMP_ERR_INVALID_ARG;
  *bytes = backward_layout(n, o).total;
  return DMP_OK;
}

int dm_purify_backward(const double* H, int64_t n, int64_t n_occ, const dmp_opts* opts, const void* tape,
                       size_t tape_bytes, const double* dLdP, double* dLdH, void* ws, size_t ws_bytes,
                       void* stream) {
  Opts o;
  int rc = normalize(opts, o);
  if (rc != DMP_OK) return rc;
  if (o.method != DMP_METHOD_PM || o.refine != 0 || o.store32) return DMP_ERR_UNSUPPORTED;  // canonical tapes only
  if (H == nullptr || tape == nullptr || dLdP == nullptr || dLdH == nullptr || ws == nullptr)
    return DMP_ERR_INVALID_ARG;
  if (n < 2 || n_occ <= 0 || n_occ >= n) return DMP_ERR_INVALID_ARG;
  const TapeLayout TL = tape_layout(n, o);
  if (tape_bytes < TL.total) return DMP_ERR_WORKSPACE;
  const BackwardLayout B = backward_layout(n, o);
  if (ws_bytes < B.total) return DMP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // ---- what the forward recorded
  TapeHeader hd;
  DMP_CUDA(cudaMemcpyAsync(&hd, static_cast<const char*>(tape) + TL.header, sizeof(hd), cudaMemcpyDeviceToHost, st));
  std::vector<double> cs(static_cast<size_t>(o.max_iter) + 1, 0.0);
  DMP_CUDA(cudaMemcpyAsync(cs.data(), static_cast<const char*>(tape) + TL.coeffs, cs.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  if (hd.magic != kTapeMagic || hd.n != n || hd.every != o.every || hd.mode != o.mode ||
      (o.mode != DMP_FP64 && (hd.s != o.s || hd.executor != o.executor)))
    return DMP_ERR_INVALID_ARG;
  if (hd.status < 0) return hd.status;
  const int K = hd.iters;
  const double* ckpt = reinterpret_cast<const double*>(static_cast<const char*>(tape) + TL.ckpt);
  const size_t nn = static_cast<size_t>(n) * n;

  double* G = reinterpret_cast<double*>(at(ws, B.G));
  double* Gn = reinterpret_cast<double*>(at(ws, B.Gn));
  double* Y = reinterpret_cast<double*>(at(ws, B.Y));
  double* Z = reinterpret_cast<double*>(at(ws, B.Z));
  double* YP = reinterpret_cast<double*>(at(ws, B.YP));
  double* ZP = reinterpret_cast<double*>(at(ws, B.ZP));
  double* segP = reinterpret_cast<double*>(at(ws, B.segP));
  double* segX = reinterpret_cast<double*>(at(ws, B.segX));
  PurifyState* state = reinterpret_cast<PurifyState*>(at(ws, B.state));
  AdjScalars* sc = reinterpret_cast<AdjScalars*>(at(ws, B.scalars));
  P0Adjoint* p0s = reinterpret_cast<P0Adjoint*>(at(ws, B.p0));
  double* part = reinterpret_cast<double*>(at(ws, B.partials));
  int* err = reinterpret_cast<int*>(at(ws, B.err));
  int32_t* expsP = reinterpret_cast<int32_t*>(at(ws, B.expsP));
  int32_t* expsA = reinterpret_cast<int32_t*>(at(ws, B.expsA));
  void* planesP = o.mode != DMP_FP64 ? at(ws, B.planesP) : nullptr;
  void* planesA = o.mode != DMP_FP64 ? at(ws, B.planesA) : nullptr;
  double* scratch = B.scratch ? reinterpret_cast<double*>(at(ws, B.scratch)) : nullptr;
  void* split_ws = B.split ? at(ws, B.split) : nullptr;
  DMP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int64_t npad = B.n_pad, kpad = B.k_pad;

  // C = A P (P symmetric; its planes are already in planesP for the Ozaki modes)
  auto times_P = [&](const double* A, const double* Pk, double* C) -> cudaError_t {
    EpiArgs e{};
    e.kind = EPI_STORE;
    e.C = C;
    e.ldc = n;
    if (o.mode == DMP_FP64) return launch_gemm_f64(A, n, Pk, n, n, n, n, 0, e, nullptr, st);
    cudaError_t r = launch_split_rows(A, n, n, n, o.s, o.beta, expsA, planesA, npad, kpad, elem_kind(o),
                                      nullptr, nullptr, st);
    if (r != cudaSuccess) return r;
    return launch_product(o, planesA, planesP, expsA, expsP, n, n, npad, npad, kpad, 0, e, nullptr,
                          err, scratch, split_ws, st);
  };
  auto split_P = [&](const double* Pk) -> cudaError_t {
    if (o.mode == DMP_FP64) return cudaSuccess;
    return launch_split_rows(Pk, n, n, n, o.s, o.beta, expsP, planesP, npad, kpad, elem_kind(o), nullptr,
                             nullptr, st);
  };

  // host copies of the per-step update weights (kept alive until the stream syncs)
  std::vector<PurifyState> wts(static_cast<size_t>(std::max(K, 1)));
  for (int k = 0; k < K; ++k) {
    std::memset(&wts[k], 0, sizeof(PurifyState));
    const double c = cs[k];
    if (c >= 0.5) {
      wts[k].alpha = 0.0;
      wts[k].b2 = (1.0 + c) / c;
      wts[k].b3 = -1.0 / c;
    } else {
      wts[k].alpha = (1.0 - 2.0 * c) / (1.0 - c);
      wts[k].b2 = (1.0 + c) / (1.0 - c);
      wts[k].b3 = -1.0 / (1.0 - c);
    }
  }

  DMP_CUDA(launch_sym_part(dLdP, n, n, G, st));
  const int E = o.every;
  for (int seg = K > 0 ? (K - 1) / E : -1; seg >= 0; --seg) {
    const int k0 = seg * E;
    const int k1 = std::min(k0 + E, K);
    // ---- recompute P_k0 .. P_{k1-1} and their squares from the checkpoint
    DMP_CUDA(cudaMemcpyAsync(segP, ckpt + static_cast<size_t>(seg) * nn, nn * sizeof(double),
                             cudaMemcpyDeviceToDevice, st));
    for (int k = k0; k < k1; ++k) {
      double* Pk = segP + static_cast<size_t>(k - k0) * nn;
      double* Xk = segX + static_cast<size_t>(k - k0) * nn;
      EpiArgs e2{};
      e2.kind = EPI_SYM_STORE;
      e2.C = Xk;
      e2.ldc = n;
      if (o.mode == DMP_FP64) {
        DMP_CUDA(launch_gemm_f64(Pk, n, Pk, n, n, n, n, 1, e2, nullptr, st));
      } else {
        DMP_CUDA(split_P(Pk));
        DMP_CUDA(launch_product(o, planesP, planesP, expsP, expsP, n, n, npad, npad, kpad, 1, e2, nullptr,
                                err, scratch, split_ws, st));
      }
      if (k + 1 < k1) {
        DMP_CUDA(cudaMemcpyAsync(&state->alpha, &wts[k].alpha, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
        EpiArgs e3{};
        e3.kind = EPI_PM_UPDATE;
        e3.C = Pk + nn;
        e3.ldc = n;
        e3.P = Pk;
        e3.ldp = n;
        e3.X2 = Xk;
        e3.ldx = n;
        e3.state = state;
        if (o.mode == DMP_FP64) {
          DMP_CUDA(launch_gemm_f64(Pk, n, Xk, n, n, n, n, 1, e3, nullptr, st));
        } else {
          DMP_CUDA(launch_split_rows(Xk, n, n, n, o.s, o.beta, expsA, planesA, npad, kpad, elem_kind(o),
                                     nullptr, nullptr, st));
          DMP_CUDA(launch_product(o, planesP, planesA, expsP, expsA, n, n, npad, npad, kpad, 1, e3, nullptr,
                                  err, scratch, split_ws, st));
        }
      }
    }
    // ---- reverse through the segment
    for (int k = k1 - 1; k >= k0; --k) {
      const double* Pk = segP + static_cast<size_t>(k - k0) * nn;
      const double* Xk = segX + static_cast<size_t>(k - k0) * nn;
      DMP_CUDA(split_P(Pk));
      DMP_CUDA(times_P(G, Pk, Y));    // Y = G P
      DMP_CUDA(launch_transpose(Y, n, n, n, Z, st));  // Z = Y^T = P G
      DMP_CUDA(times_P(Y, Pk, YP));   // G P^2
      DMP_CUDA(times_P(Z, Pk, ZP));   // P G P
      DMP_CUDA(launch_adj_reduce(Pk, Xk, G, Z, n, part, cs[k], sc, st));
      DMP_CUDA(launch_adj_step(G, Y, YP, ZP, Pk, Xk, n, sc, Gn, st));
      std::swap(G, Gn);
    }
    int flag = 0;
    DMP_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DMP_CUDA(cudaStreamSynchronize(st));
    if (flag) return DMP_ERR_TIMEOUT;
  }
  // ---- through the initial guess
  P0Adjoint h0;
  std::memset(&h0, 0, sizeof(h0));
  h0.n = static_cast<double>(n);
  h0.n_occ = static_cast<double>(n_occ);
  h0.lam = hd.lam;
  h0.mu = hd.mu;
  h0.h_min = hd.h_min;
  h0.h_max = hd.h_max;
  h0.lam_branch = hd.lam_branch;
  h0.row_min = hd.row_min;
  h0.row_max = hd.row_max;
  h0.bounds_grad = (opts->flags & DMP_FLAG_BOUNDS_CONSTANT) ? 0 : 1;
  DMP_CUDA(cudaMemcpyAsync(p0s, &h0, sizeof(h0), cudaMemcpyHostToDevice, st));
  DMP_CUDA(launch_p0_adjoint(G, H, n, n, part, p0s, dLdH, n, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  return DMP_OK;
}

int dm_foe_workspace_size(int64_t n, const dmp_foe_params* params, const dmp_opts* opts, size_t* bytes) {
  Opts o;
  const int rc = foe_opts(opts, o);
  if (rc != DMP_OK) return rc;
  if (n < 2 || bytes == nullptr || params == nullptr) return DMP_ERR_INVALID_ARG;
  const int M = params->n_terms;
  const int scheme = params->scheme;
  if (M < 2 || M > kFoeMaxTerms) return DMP_ERR_INVALID_ARG;
  if (scheme != DMP_FOE_RECURRENCE && scheme != DMP_FOE_PATERSON_STOCKMEYER) return DMP_ERR_INVALID_ARG;
  *bytes = foe_layout(n, o, scheme, M).total;
  return DMP_OK;
}

int dm_foe(const double* H, int64_t n, int64_t ldh, const dmp_foe_params* params, const dmp_opts* opts,
           double* P, int64_t ldp, dmp_foe_info* info, void* ws, size_t ws_bytes, void* stream) {
  Opts o;
  int rc = foe_opts(opts, o);
  if (rc != DMP_OK) return rc;
  if (H == nullptr || P == nullptr || ws == nullptr || params == nullptr) return DMP_ERR_INVALID_ARG;
  if (n < 2 || ldh < n || ldp < n) return DMP_ERR_INVALID_ARG;
  const dmp_foe_params fp = *params;
  const int M = fp.n_terms;
  const bool canonical = fp.n_occ > 0;
  const bool ps = fp.scheme == DMP_FOE_PATERSON_STOCKMEYER;
  if (!(fp.kT > 0.0) || !std::isfinite(fp.kT)) return DMP_ERR_INVALID_ARG;
  if (fp.n_occ < 0 || fp.n_occ >= n) return DMP_ERR_INVALID_ARG;
  if (!canonical && !std::isfinite(fp.mu)) return DMP_ERR_INVALID_ARG;
  if (M < 2 || M > kFoeMaxTerms) return DMP_ERR_INVALID_ARG;
  if (fp.scheme != DMP_FOE_RECURRENCE && !ps) return DMP_ERR_INVALID_ARG;
  if (!std::isfinite(fp.e_min) || !std::isfinite(fp.e_max)) return DMP_ERR_INVALID_ARG;
  if (o.mode != DMP_FP64 && !levels_fit_int32(n, o.s, o.mode)) return DMP_ERR_UNSUPPORTED;
  const FoeLayout L = foe_layout(n, o, fp.scheme, M);
  if (ws_bytes < L.total) return DMP_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  auto dbl = [&](size_t off) { return reinterpret_cast<double*>(at(ws, off)); };
  PurifyState* state = reinterpret_cast<PurifyState*>(at(ws, L.state));
  double* rowbuf = dbl(L.rowbuf);
  FoeScalars* sc = reinterpret_cast<FoeScalars*>(at(ws, L.scal));
  double* coeffs = dbl(L.coeffs);
  double* traces = dbl(L.traces);
  double* w = dbl(L.w);
  double* gx = dbl(L.gx);
  double* partials = dbl(L.partials);
  int* err = reinterpret_cast<int*>(at(ws, L.err));
  double* Hs = dbl(L.Hs);
  double* Ta = dbl(L.Ta);
  double* Tb = dbl(L.Tb);
  double* Y = dbl(L.Y);
  const bool oz = o.mode != DMP_FP64;
  int32_t* expsH = oz ? reinterpret_cast<int32_t*>(at(ws, L.expsH)) : nullptr;
  int32_t* expsT = oz ? reinterpret_cast<int32_t*>(at(ws, L.expsT)) : nullptr;
  void* planesH = oz ? at(ws, L.planesH) : nullptr;
  void* planesT = oz ? at(ws, L.planesT) : nullptr;
  double* scratch = L.scratch ? dbl(L.scratch) : nullptr;
  void* split_ws = L.split ? at(ws, L.split) : nullptr;
  DMP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));

  PurifyState init;
  std::memset(&init, 0, sizeof(init));
  DMP_CUDA(cudaMemcpyAsync(state, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  // Gershgorin bounds and the NaN/Inf check of H (the canonical initial guess
  // this pass also writes into P is overwritten below)
  DMP_CUDA(launch_gershgorin_init(H, n, ldh, canonical ? fp.n_occ : n / 2, rowbuf, state, P, ldp, st));
  DMP_CUDA(launch_foe_scale(state, fp.e_min, fp.e_max, fp.e_min < fp.e_max ? 1 : 0, sc, st));
  int32_t nonfinite = 0;
  DMP_CUDA(cudaMemcpyAsync(&nonfinite, &sc->nonfinite, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  if (nonfinite) {
    if (info != nullptr) {
      std::memset(info, 0, sizeof(*info));
      info->status = DMP_ERR_NONFINITE;
    }
    return DMP_ERR_NONFINITE;
  }

  int products = 0;
  // Symmetric product Y = A B of two polynomials in H_s: A's digit planes
  // (pa, ea) are prepared by the caller, B is split here (FP64: A itself).
  // After a product whose bounded device wait ran out, the error flag makes
  // every later split and product kernel return at once (it is their `done`
  // word), and every kFoeCheckEvery products the host reads the flag and
  // stops enqueueing with DMP_ERR_TIMEOUT.
  constexpr int kFoeCheckEvery = 8;
  auto product = [&](const double* A, const void* pa, const int32_t* ea, const double* B) -> int {
    EpiArgs e{};
    e.kind = EPI_SYM_STORE;
    e.C = Y;
    e.ldc = n;
    if (!oz) {
      DMP_CUDA(launch_gemm_f64(A, n, B, n, n, n, n, 1, e, nullptr, st));
    } else {
      DMP_CUDA(launch_split_rows(B, n, n, n, o.s, o.beta, expsT, planesT, L.n_pad, L.k_pad, elem_kind(o), nullptr,
                                 err, st));
      DMP_CUDA(launch_product(o, pa, planesT, ea, expsT, n, n, L.n_pad, L.n_pad, L.k_pad, 1, e, err,
                              err, scratch, split_ws, st));
    }
    ++products;
    if (oz && o.executor == DMP_EXEC_TC && products % kFoeCheckEvery == 0) {
      int32_t flag = 0;
      DMP_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      DMP_CUDA(cudaStreamSynchronize(st));
      if (flag) return DMP_ERR_TIMEOUT;
    }
    return DMP_OK;
  };
  auto split_a = [&](const double* A, void* planes, int32_t* exps) -> int {
    if (oz)
      DMP_CUDA(launch_split_rows(A, n, n, n, o.s, o.beta, exps, planes, L.n_pad, L.k_pad, elem_kind(o), nullptr,
                                 err, st));
    return DMP_OK;
  };

  if (!ps) {
    bool h_split = false;
    // One pass of T_{k+1} = 2 H_s T_k - T_{k-1}: with `acc` it forms P from the
    // coefficients, else it records tr T_k.
    auto pass = [&](bool acc) -> int {
      DMP_CUDA(launch_foe_init(H, ldh, n, sc, acc ? coeffs : nullptr, Hs, Ta, Tb, P, ldp, st));
      if (!acc) {
        DMP_CUDA(launch_foe_trace(Ta, n, n, traces, st));
        DMP_CUDA(launch_foe_trace(Tb, n, n, traces + 1, st));
      }
      if (!h_split && M > 2) {
        // H_s is the same in both passes: its digit planes serve every product
        if (split_a(Hs, planesH, expsH) != DMP_OK) return DMP_ERR_CUDA;
        h_split = true;
      }
      double* prev = Ta;
      double* cur = Tb;
      for (int k = 1; k <= M - 2; ++k) {
        const int prc = product(Hs, planesH, expsH, cur);
        if (prc != DMP_OK) return prc;
        DMP_CUDA(launch_foe_step(Y, prev, acc ? P : nullptr, ldp, coeffs + k + 1, n, st));
        if (!acc) DMP_CUDA(launch_foe_trace(prev, n, n, traces + k + 1, st));
        std::swap(prev, cur);
      }
      return DMP_OK;
    };
    if (canonical) {
      rc = pass(false);
      if (rc != DMP_OK) return rc;
      DMP_CUDA(launch_foe_coefficients(sc, fp.kT, 0.0, static_cast<double>(fp.n_occ), traces, M, w, gx, coeffs, st));
    } else {
      DMP_CUDA(launch_foe_coefficients(sc, fp.kT, fp.mu, 0.0, nullptr, M, w, gx, coeffs, st));
    }
    rc = pass(true);
    if (rc != DMP_OK) return rc;
  } else {
    // ---- Paterson-Stockmeyer scheme: baby steps T_1 .. T_nb in slots (T_1 = H_s)
    const int q = ps_q(M);
    const int r = (M + q - 1) / q;
    const int nb = r > 1 ? q : q - 1;
    double* Tps = dbl(L.Tps);
    auto slot = [&](int t) { return Tps + static_cast<size_t>(t - 1) * n * n; };
    int32_t* expsY = oz ? reinterpret_cast<int32_t*>(at(ws, L.expsY)) : nullptr;
    void* planesY = oz ? at(ws, L.planesY) : nullptr;
    double* ip = dbl(L.ip);
    double* dots = dbl(L.dots);
    double* fold = dbl(L.fold);
    double* psw = dbl(L.psw);
    DMP_CUDA(launch_foe_init(H, ldh, n, sc, nullptr, slot(1), nullptr, nullptr, P, ldp, st));
    if (nb >= 2 && split_a(slot(1), planesH, expsH) != DMP_OK) return DMP_ERR_CUDA;
    for (int j = 1; j < nb; ++j) {
      rc = product(slot(1), planesH, expsH, slot(j));
      if (rc != DMP_OK) return rc;
      DMP_CUDA(launch_foe_next(Y, j == 1 ? nullptr : slot(j - 1), slot(j + 1), n, st));
    }
    double* yq = r > 1 ? slot(q) : nullptr;
    if (r > 1 && split_a(yq, planesY, expsY) != DMP_OK) return DMP_ERR_CUDA;
    if (canonical) {
      // traces: T_1 .. T_{q-1} directly; T_{qm} = T_m(y) by the recurrence in y
      // (T_q for m = 1), with <T_{qm}, T_j> for the rest
      for (int k = 1; k < q && k < M; ++k) DMP_CUDA(launch_foe_trace(slot(k), n, n, traces + k, st));
      double* g_prev = nullptr;  // T_0 = I
      double* g_cur = yq;
      for (int m = 1; q * m < M; ++m) {
        if (m >= 2) {
          rc = product(yq, planesY, expsY, g_cur);
          if (rc != DMP_OK) return rc;
          // G_2 and G_3 take the two free buffers; later terms overwrite G_{m-2} in place
          double* out = m == 2 ? Ta : (m == 3 ? Tb : g_prev);
          DMP_CUDA(launch_foe_next(Y, g_prev, out, n, st));
          g_prev = g_cur;
          g_cur = out;
        }
        DMP_CUDA(launch_foe_trace(g_cur, n, n, traces + q * m, st));
        DMP_CUDA(launch_foe_dots(g_cur, Tps, q, n, dots, ip + static_cast<size_t>(m) * q + 1, st));
      }
      DMP_CUDA(launch_foe_ps_traces(traces, ip, q, M, n, st));
      DMP_CUDA(launch_foe_coefficients(sc, fp.kT, 0.0, static_cast<double>(fp.n_occ), traces, M, w, gx, coeffs, st));
    } else {
      DMP_CUDA(launch_foe_coefficients(sc, fp.kT, fp.mu, 0.0, nullptr, M, w, gx, coeffs, st));
    }
    DMP_CUDA(launch_foe_fold(coeffs, M, q, r, fold, psw, st));
    // Clenshaw in y: b_m = B_m + 2 y b_{m+1} - b_{m+2}, P = B_0 + y b_1 - b_2
    if (r == 1) {
      DMP_CUDA(launch_foe_combine(Tps, q, psw, nullptr, 0.0, nullptr, P, ldp, n, st));
    } else {
      double* b1 = Ta;
      double* b2 = nullptr;  // zero
      DMP_CUDA(launch_foe_combine(Tps, q, psw + static_cast<size_t>(r - 1) * q, nullptr, 0.0, nullptr, b1, n, n, st));
      for (int m = r - 2; m >= 1; --m) {
        rc = product(yq, planesY, expsY, b1);
        if (rc != DMP_OK) return rc;
        double* out = b2 ? b2 : Tb;
        DMP_CUDA(launch_foe_combine(Tps, q, psw + static_cast<size_t>(m) * q, Y, 2.0, b2, out, n, n, st));
        b2 = b1;
        b1 = out;
      }
      rc = product(yq, planesY, expsY, b1);
      if (rc != DMP_OK) return rc;
      DMP_CUDA(launch_foe_combine(Tps, q, psw, Y, 1.0, b2, P, ldp, n, st));
    }
  }
  DMP_CUDA(launch_energy(P, ldp, H, ldh, n, partials, state, st));
  DMP_CUDA(launch_foe_trace(P, ldp, n, &sc->trace, st));

  FoeScalars fin;
  double energy = 0.0;
  double last[2] = {0.0, 0.0};
  int32_t err_end = 0;
  DMP_CUDA(cudaMemcpyAsync(&fin, sc, sizeof(fin), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaMemcpyAsync(&energy, &state->energy_refined, sizeof(double), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaMemcpyAsync(last, coeffs + (M - 2), 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaMemcpyAsync(&err_end, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DMP_CUDA(cudaStreamSynchronize(st));
  if (err_end) return DMP_ERR_TIMEOUT;
  if (info != nullptr) {
    info->status = DMP_OK;
    info->n_terms = M;
    info->products = products;
    info->slices_used = o.s;
    info->mu = fin.mu;
    info->trace = fin.trace;
    info->energy = energy;
    info->band_energy = 2.0 * energy;
    info->e_min = fin.e_min;
    info->e_max = fin.e_max;
    info->tail = std::fabs(last[0]) + std::fabs(last[1]);
  }
  return DMP_OK;
}

}  // extern "C"
