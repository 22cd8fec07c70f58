// Internal declarations shared by the libdmp translation units.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; no driver library is linked)
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/dmp.h"

namespace dmp {

// ---------------------------------------------------------------- constants
constexpr int kMaxSlices = 12;   // beta 7: up to 10 (70 bits); beta 8: 9 (72); beta 5 nearest: 12 (60)
constexpr int kTileM = 128;      // output tile rows of the slice-pair GEMMs
constexpr int kTileN = 128;      // output tile columns
constexpr int kPadK = 128;       // digit planes are padded to a multiple of this along K (two
                                 // 64-element swizzle atoms: the paired tcgen05 kernel stages 128)
constexpr int kPadK8 = 256;      // the same for one-byte E4M3 digits (two 128-element atoms)
constexpr int32_t kBadExp = 0x7fffffff;  // row exponent of a row holding NaN/Inf

inline int beta_of(int mode) { return mode == DMP_OZAKI_BF16 ? 8 : (mode == DMP_OZAKI_E4M3 ? 5 : 7); }
// largest digit magnitude: 127 for the truncated INT8 digits, 2^(beta-1) for
// the nearest digits (E4M3: 16, BF16: 128)
inline int digit_max(int mode) {
  return mode == DMP_OZAKI_E4M3 ? 16 : (mode == DMP_OZAKI_BF16 ? 128 : 127);
}
// largest slice count: 70 bits (beta 7), 72 (beta 8), 60 (E4M3 nearest digits)
inline int max_slices(int mode) { return mode == DMP_OZAKI_E4M3 ? 12 : (mode == DMP_OZAKI_BF16 ? 9 : 10); }
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------- launch accounting
extern std::atomic<long long> g_launches;
inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------- device-side run state
// One per purification. Written by the measurement kernel, read by the update
// epilogue and the host.
struct PurifyState {
  // measures of the current iterate P_k
  double t1, t2, t3, idem2, energy;
  // band-energy history (Tr(HK) of the last three iterates, newest first)
  double band[3];
  // coefficient and update weights P' = alpha P + b2 P^2 + b3 P^3
  double c, alpha, b2, b3;
  // initial-guess scalars
  double h_min, h_max, mu, lam;
  int32_t row_min, row_max, lam_branch;
  int32_t iter;     // updates applied so far
  int32_t status;   // DMP_* code once done
  int32_t done;     // nonzero once a stopping rule fired (kernels then skip work)
  int32_t nonfinite;
  int32_t branch;   // 1: c >= 1/2, 2: c < 1/2
  // tr(P' H) of the refined matrix (refinement step only)
  double energy_refined;
  // method (DMP_METHOD_*) and the per-step data of SP2 / TRS4
  int32_t method;
  int32_t step_kind;      // 0: X' = alpha X + b2 X2 (elementwise); 1: X' = X2 Z (TRS4 product)
  double t4;              // tr X^4 = ||X2||_F^2
  double idem_hist[3];    // ||X2 - X||_F of the last three iterates, newest first
  double zd, zx, zx2;     // TRS4: Z = zd I + zx X + zx2 X2
  double n_occ_d;         // n_occ
  double p0_scale, p0_shift;  // initial guess -p0_scale H + p0_shift I (canonical: built as in the method)
  // options copied for the device
  double tol, energy_tol;
  int32_t max_iter;
  int32_t store32;  // DMP_FLAG_FP32_STORAGE: stored matrices rounded to FP32 values
};

// A matrix element as it is stored: rounded to the nearest FP32 value under
// DMP_FLAG_FP32_STORAGE (round to nearest even, subnormals kept), else as is.
__device__ __forceinline__ double stored_value(double v, bool round32) {
  return round32 ? static_cast<double>(__double2float_rn(v)) : v;
}

// ---------------------------------------------------------------- kernels (host launchers)
// All launchers return cudaSuccess or the launch error; they count launches.

// Row split: exponents e_r and `s` digit planes of beta bits of the m x k matrix
// A (leading dimension lda). Planes are [s][m_pad][k_pad], element kind 1
// (int8 truncated digits), 3 (bfloat16: the beta 7 truncated digits, or the
// beta 8 nearest digits) or 4 (beta 5 nearest digits as E4M3 bytes). Nearest
// digits take a row exponent one larger. Padding rows/columns are zero. Sets
// *flag to 1 if A holds a NaN/Inf.
cudaError_t launch_split_rows(const double* A, int64_t m, int64_t k, int64_t lda, int s, int beta,
                              int32_t* exps, void* planes, int64_t m_pad, int64_t k_pad,
                              int elem_kind, int* flag, const int* done, cudaStream_t st);

// Out-of-place transpose (m x n, lda) -> (n x m, leading dimension m).
cudaError_t launch_transpose(const double* A, int64_t m, int64_t n, int64_t lda, double* At,
                             cudaStream_t st);

enum EpiKind { EPI_STORE = 0, EPI_SYM_STORE = 1, EPI_PM_UPDATE = 2, EPI_LEVELS = 3 };

struct EpiArgs {
  int kind;
  double* C;          // output (EPI_STORE / EPI_SYM_STORE / EPI_PM_UPDATE: P_next)
  int64_t ldc;
  const double* P;    // EPI_PM_UPDATE: current iterate
  const double* X2;   // EPI_PM_UPDATE: P^2
  int64_t ldp;        // leading dimension of P
  int64_t ldx;        // leading dimension of X2
  const PurifyState* state;  // EPI_PM_UPDATE weights
  int32_t* levels;    // EPI_LEVELS: [s][m][n]
  int round32;        // round every stored element to an FP32 value (DMP_FLAG_FP32_STORAGE)
};

// IMMA executor: level sums of int8 planes with fused FP64 recombination.
// sym != 0 computes only the tiles on and above the diagonal (m == n, B planes
// are the transposed operand of a symmetric product) and mirrors them.
cudaError_t launch_ozaki_imma(const int8_t* A, const int8_t* B, const int32_t* ea, const int32_t* eb,
                              int64_t m, int64_t n, int64_t m_pad, int64_t n_pad, int64_t k_pad,
                              int s, int beta, int sym, const EpiArgs& epi, const int* done,
                              cudaStream_t st);

// tcgen05 executor (bf16-carried digits, TMEM accumulators, TMA operands).
// A planes [s][rows_a][k_pad], B planes [s][rows_b][k_pad] in bfloat16 (E4M3
// bytes for beta 5); rows_a a multiple of 128, rows_b of 256, k_pad of 64
// (128 for beta 5).
// *err is set to 1 if a bounded device wait expired. `scratch` holds
// tc_scratch_bytes() of per-CTA float64 partial sums (the kernel is persistent:
// at most kTcMaxCtas CTAs, one per SM).
constexpr int kTcMaxCtas = 160;
size_t tc_scratch_bytes();
// workspace of the tcgen05 executor's split launches (the tiles' shared group sums and
// counters); a launch given none runs whole tiles only
size_t tc_split_bytes();
// whether single-matrix tcgen05 products that fill at most half a wave of CTAs
// are split into chunk units shared by every CTA; returns the previous setting
int set_tc_split_tiles(int enable);
// beta = 7 single-matrix products on CTA pairs (2-SM MMA); returns the previous setting
int set_tc_pairing(int enable);
// whether products may run on CTA pairs (the pairing switch is on and clusters of
// two CTAs of the paired kernel can be resident)
bool tc_pairs_available();
// The next tcgen05 product launch withholds each CTA's first operand stage and
// bounds its waits by wait_limit_us (the bounded-wait test); one-shot.
int set_stall_test(int wait_limit_us);
cudaError_t launch_ozaki_tc(const void* A, const void* B, const int32_t* ea, const int32_t* eb, int64_t m,
                            int64_t n, int64_t rows_a, int64_t rows_b, int64_t k_pad, int s, int beta, int sym,
                            const EpiArgs& epi, const int* done, int* err, double* scratch, void* split_ws,
                            cudaStream_t st);

// FP64 executor: C = A B (A m x k, B k x n row-major) with the same epilogues.
cudaError_t launch_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m,
                            int64_t n, int64_t k, int sym, const EpiArgs& epi, const int* done,
                            cudaStream_t st);

// Purification support kernels.
cudaError_t launch_gershgorin_init(const double* H, int64_t n, int64_t ldh, int64_t n_occ,
                                   double* rowbuf, PurifyState* state, double* P, int64_t ldp,
                                   cudaStream_t st);
size_t gershgorin_rowbuf_bytes(int64_t n);
// Refinement step: the update weights of c = 1/2 (P' = 3 P^2 - 2 P^3), and
// state->energy_refined = tr(P H) (deterministic, from the upper triangles).
cudaError_t launch_refine_weights(PurifyState* state, cudaStream_t st);
cudaError_t launch_energy(const double* P, int64_t ldp, const double* H, int64_t ldh, int64_t n, double* partials,
                          PurifyState* state, cudaStream_t st);
// SP2 / TRS4: measures with tr X^4 and variant_decide; the elementwise step
// Out = alpha X + b2 X2; the TRS4 factor Z = zd I + zx X + zx2 X2 (weights from
// the state; full n x n, so the results are exactly symmetric as X and X2 are).
cudaError_t launch_measure_variant(const double* X, int64_t ldx, const double* X2, int64_t ldx2, const double* H,
                                   int64_t ldh, int64_t n, double* partials, PurifyState* state, cudaStream_t st);
cudaError_t launch_axpby(const double* X, int64_t ldx, const double* X2, int64_t ldx2, double* out, int64_t ldo,
                         int64_t n, const PurifyState* state, cudaStream_t st);
cudaError_t launch_trs4_z(const double* X, int64_t ldx, const double* X2, int64_t ldx2, double* out, int64_t ldo,
                          int64_t n, const PurifyState* state, cudaStream_t st);
cudaError_t launch_measure(const double* P, int64_t ldp, const double* X2, int64_t ldx,
                           const double* H, int64_t ldh, int64_t n, double* partials,
                           PurifyState* state, cudaStream_t st);
cudaError_t launch_copy_matrix(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t m,
                               int64_t n, cudaStream_t st);

constexpr int kMeasureBlocks = 608;  // 4 x 152 SMs; fixed so sums are reproducible

// Chebyshev Fermi-operator expansion (csrc/foe.cu). Scalars on the device:
// the enclosure [e_min, e_max] that scales H, its centre a and half-width b,
// the chemical potential and the trace of the result.
struct FoeScalars {
  double a, b, mu, e_min, e_max, trace;
  int32_t nonfinite;  // H held a NaN/Inf (copied from the Gershgorin pass)
};
constexpr int kFoeMaxTerms = 16384;  // DMP_FOE_MAX_TERMS
// Enclosure: the given one when use_given, else the Gershgorin bounds in `state`.
cudaError_t launch_foe_scale(const PurifyState* state, double e_min, double e_max, int use_given, FoeScalars* sc,
                             cudaStream_t st);
// mu (solved from n_occ and the traces tr T_k when `traces` is non-null, else
// the given mu), then the M coefficients. w and gx hold 2M doubles each.
cudaError_t launch_foe_coefficients(FoeScalars* sc, double kT, double mu, double n_occ, const double* traces, int M,
                                    double* w, double* gx, double* coeffs, cudaStream_t st);
// H_s, T_0 = I, T_1 = H_s (leading dimension n) and, with coeffs, P = c_0/2 I + c_1 H_s.
cudaError_t launch_foe_init(const double* H, int64_t ldh, int64_t n, const FoeScalars* sc, const double* coeffs,
                            double* Hs, double* T0, double* T1, double* P, int64_t ldp, cudaStream_t st);
// Tprev <- 2 Y - Tprev; with P non-null, P += (*coeff) Tprev.
cudaError_t launch_foe_step(const double* Y, double* Tprev, double* P, int64_t ldp, const double* coeff, int64_t n,
                            cudaStream_t st);
// *out = tr A (fixed order).
cudaError_t launch_foe_trace(const double* A, int64_t lda, int64_t n, double* out, cudaStream_t st);
// Paterson-Stockmeyer scheme. Baby steps T_1 .. T_q are kept in consecutive
// n x n slots (T_t at T + (t - 1) n^2; T_0 = I implicit).
constexpr int kFoeDotBlocks = 304;  // 2 x 152 SMs; fixed so sums are reproducible
// Tout = 2 Y - Tprev (Tprev = I when null; Tout may be Tprev).
cudaError_t launch_foe_next(const double* Y, const double* Tprev, double* Tout, int64_t n, cudaStream_t st);
// out = ((w_0 I + sum_{t=1}^{nt-1} w_t T_t) + alpha Y) - Bm2 (Y, Bm2 nullable; out
// of leading dimension ldo may be Bm2).
cudaError_t launch_foe_combine(const double* T, int nt, const double* w, const double* Y, double alpha,
                               const double* Bm2, double* out, int64_t ldo, int64_t n, cudaStream_t st);
// out[t - 1] = <G, T_t>_F for t = 1 .. nt - 1; partials holds kFoeDotBlocks (nt - 1) doubles.
cudaError_t launch_foe_dots(const double* G, const double* T, int nt, int64_t n, double* partials, double* out,
                            cudaStream_t st);
// tr T_k, k < M, from the baby- and giant-step traces already in `traces` and the
// Frobenius products ip[m q + j] = <T_{qm}, T_j>.
cudaError_t launch_foe_ps_traces(double* traces, const double* ip, int q, int M, int64_t n, cudaStream_t st);
// Block weights w[r][q] from the M coefficients (a: scratch of r q doubles).
cudaError_t launch_foe_fold(const double* coeffs, int M, int q, int r, double* a, double* w, cudaStream_t st);

}  // namespace dmp

namespace dmp {

// ---------------------------------------------------------------- shared epilogue
// Applies one output element v = C[r][c] of a product. `mirror` writes the
// transposed element as well (off-diagonal tiles of a symmetric product).
__device__ __forceinline__ void epi_apply(const EpiArgs& e, int64_t r, int64_t c, double v,
                                          bool mirror) {
  if (e.kind == EPI_PM_UPDATE) {
    const double p = e.P[r * e.ldp + c];
    const double x2 = e.X2[r * e.ldx + c];
    v = e.state->alpha * p + e.state->b2 * x2 + e.state->b3 * v;
  }
  v = stored_value(v, e.round32 != 0);
  e.C[r * e.ldc + c] = v;
  if (mirror) e.C[c * e.ldc + r] = v;
}

// Upper-triangle tile enumeration: tile index -> (bi, bj) with bi <= bj, row-major.
__device__ __forceinline__ void upper_tile(int idx, int T, int& bi, int& bj) {
  int b = 0;
  int start = 0;
  while (start + (T - b) <= idx) {
    start += T - b;
    ++b;
  }
  bi = b;
  bj = b + (idx - start);
}

}  // namespace dmp

namespace dmp {

// Brackets one launch with profiling events when dmp_profile_enable(1) is on.
class ProfScope {
 public:
  ProfScope(int kind, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  int idx_;
};

}  // namespace dmp

namespace dmp {

// ---------------------------------------------------------------- adjoint
struct AdjScalars {
  double alpha, b2, b3, td, tn, dLdc;
};

struct P0Adjoint {
  double n, n_occ, lam, mu, h_min, h_max;
  int32_t lam_branch, row_min, row_max, bounds_grad;
  double diag_add, dhmax, dhmin;  // written on the device
};

cudaError_t launch_adj_reduce(const double* P, const double* X2, const double* G, const double* Z, int64_t n,
                              double* part, double c, AdjScalars* sc, cudaStream_t st);
cudaError_t launch_adj_step(const double* G, const double* Y, const double* YP, const double* ZP,
                            const double* P, const double* X2, int64_t n, const AdjScalars* sc, double* Gn,
                            cudaStream_t st);
cudaError_t launch_sym_part(const double* A, int64_t ld, int64_t n, double* out, cudaStream_t st);
cudaError_t launch_p0_adjoint(const double* G0, const double* H, int64_t ldh, int64_t n, double* part,
                              P0Adjoint* s, double* out, int64_t ldo, cudaStream_t st);

}  // namespace dmp

namespace dmp {

// ---------------------------------------------------------------- batched purification
// One descriptor per matrix of a batch, in device memory. The tcgen05 tensor
// maps of its digit planes live here (global memory), so that one grouped
// launch can serve tiles of every matrix.
struct alignas(128) BatchMat {
  CUtensorMap tmPa;   // planes of P, 128-row boxes (A operand)
  CUtensorMap tmPb;   // planes of P, BN-row boxes (B operand of P P)
  CUtensorMap tmXb;   // planes of X2, BN-row boxes (B operand of P X2)
  double* buf[2];     // iterates: buf[0] is the caller's P, buf[1] a workspace copy
  double* X2;
  const double* H;
  void* planesP;
  void* planesX;
  int32_t* expsP;
  int32_t* expsX;
  PurifyState* state;
  int64_t n, n_occ, ldh, ldp, n_pad, k_pad;
  int32_t s, pad_;
};

// 2-D TMA map over s stacked bf16 digit planes (k_pad contiguous, rows_total
// rows), 64 x box_rows boxes with 128-byte swizzle.
bool make_plane_map_ext(CUtensorMap* tm, const void* planes, int64_t k_pad, int64_t rows_total, int box_rows,
                        bool f8);

// Grouped kernels (every launch covers all matrices; finished ones are skipped).
// `which`: 0 = buf[0], 1 = buf[1], 2 = X2.
cudaError_t launch_split_grouped(const BatchMat* mats, const int64_t* row_start, int nmats, int64_t total_rows,
                                 int which, int beta, int s, cudaStream_t st);
cudaError_t launch_measure_grouped(const BatchMat* mats, int nmats, int cur, double* partials,
                                   cudaGraphConditionalHandle cond, int set_cond, int* active,
                                   cudaStream_t st);
cudaError_t launch_finish_grouped(const BatchMat* mats, int nmats, cudaStream_t st);
// phase 0: X2 = P P from buf[cur]; phase 1: update buf[cur] -> buf[1 - cur].
// `counter` (one int of device memory) is zeroed on the stream before a
// single-CTA launch; its CTAs take tiles from it in list order.
// `pair`: CTA pairs on 256-row tiles (bn 256; the tiles' row blocks are 256
// rows and the B maps have bn / 2-row boxes), else single CTAs on 128-row tiles.
cudaError_t launch_ozaki_tc_grouped(const BatchMat* mats, const int4* tiles, int ntiles, int bn, bool pair, int beta,
                                    int phase, int cur, int* err, double* scratch, int* counter, cudaStream_t st);

}  // namespace dmp

namespace dmp {

// The stopping rules and the coefficient of canonical purification, applied to
// the measures of the current iterate (diagonal/strict-upper partial sums:
// tot = {tr P, tr X2, diag PX2, upper PX2, diag (X2-P)^2, upper (X2-P)^2,
// diag PH, upper PH}). Sets status/done, or c and the update weights.
// (SP2 / TRS4 use variant_decide below.)
__device__ __forceinline__ void pm_decide(PurifyState* st, const double* tot) {
  const double t1 = tot[0], t2 = tot[1];
  const double t3 = tot[2] + 2.0 * tot[3];
  const double idem2 = tot[4] + 2.0 * tot[5];
  const double energy = tot[6] + 2.0 * tot[7];
  st->t1 = t1;
  st->t2 = t2;
  st->t3 = t3;
  st->idem2 = idem2;
  st->energy = energy;
  if (!isfinite(t1) || !isfinite(t2) || !isfinite(t3) || !isfinite(idem2) || !isfinite(energy)) {
    st->nonfinite = 1;
    st->status = DMP_ERR_NONFINITE;
    st->done = 1;
    return;
  }
  const int k = st->iter;
  st->band[2] = st->band[1];
  st->band[1] = st->band[0];
  st->band[0] = 2.0 * energy;
  const double idem = sqrt(idem2);
  if (idem < st->tol) {
    st->status = DMP_OK;
    st->done = 1;
    return;
  }
  const double b0 = st->band[0], b1 = st->band[1], b2 = st->band[2];
  if (k >= 2 && b0 > b1 && b1 > b2 && fabs(b0 - b1) < 1e-2 && fabs(b1 - b2) < 1e-2) {
    st->status = DMP_STALLED;
    st->done = 1;
    return;
  }
  if (st->energy_tol > 0.0 && k >= 1 && fabs(b0 - b1) < st->energy_tol) {
    st->status = DMP_OK;
    st->done = 1;
    return;
  }
  if (k >= st->max_iter) {
    st->status = DMP_NOT_CONVERGED;
    st->done = 1;
    return;
  }
  const double td = t1 - t2;
  if (!(td > 0.0)) {
    st->status = DMP_C_OUT_OF_RANGE;
    st->done = 1;
    return;
  }
  const double c = (t2 - t3) / td;
  if (!(c >= 0.0 && c <= 1.0)) {
    st->status = DMP_C_OUT_OF_RANGE;
    st->done = 1;
    return;
  }
  st->c = c;
  if (c >= 0.5) {
    st->alpha = 0.0;
    st->b2 = (1.0 + c) / c;
    st->b3 = -1.0 / c;
    st->branch = 1;
  } else {
    st->alpha = (1.0 - 2.0 * c) / (1.0 - c);
    st->b2 = (1.0 + c) / (1.0 - c);
    st->b3 = -1.0 / (1.0 - c);
    st->branch = 2;
  }
  st->iter = k + 1;
}

// SP2 / TRS4 stopping rules and step (the cited recursions; readings as in the
// oracle): tot as for pm_decide plus {diag X2^2, upper X2^2}. Rules on X_k:
// ||X2 - X|| < tol -> DMP_OK; k >= 2, the value two steps earlier below 1 and
// not above the current one -> DMP_C_OUT_OF_RANGE (rounding floor); k ==
// max_iter -> DMP_NOT_CONVERGED. Else the step: SP2 squares or takes 2X - X2,
// whichever brings the trace closer to n_occ; TRS4 takes gamma = (n_occ - tr F)
// / tr G with tr F = 4 tr X^3 - 3 tr X^4 and tr G = ||X2 - X||^2, SP2 steps for
// gamma outside [0, 6], else X' = X2 Z. c is gamma (TRS4) or 1 / 0 for a
// squaring / 2X - X2 step (SP2).
__device__ __forceinline__ void variant_decide(PurifyState* st, const double* tot) {
  const double t1 = tot[0], t2 = tot[1];
  const double t3 = tot[2] + 2.0 * tot[3];
  const double idem2 = tot[4] + 2.0 * tot[5];
  const double energy = tot[6] + 2.0 * tot[7];
  const double t4 = tot[8] + 2.0 * tot[9];
  st->t1 = t1;
  st->t2 = t2;
  st->t3 = t3;
  st->t4 = t4;
  st->idem2 = idem2;
  st->energy = energy;
  if (!isfinite(t1) || !isfinite(t2) || !isfinite(t3) || !isfinite(t4) || !isfinite(idem2) ||
      !isfinite(energy)) {
    st->nonfinite = 1;
    st->status = DMP_ERR_NONFINITE;
    st->done = 1;
    return;
  }
  const int k = st->iter;
  const double idem = sqrt(idem2);
  st->idem_hist[2] = st->idem_hist[1];
  st->idem_hist[1] = st->idem_hist[0];
  st->idem_hist[0] = idem;
  if (idem < st->tol) {
    st->status = DMP_OK;
    st->done = 1;
    return;
  }
  if (k >= 2 && st->idem_hist[2] < 1.0 && idem >= st->idem_hist[2]) {
    st->status = DMP_C_OUT_OF_RANGE;
    st->done = 1;
    return;
  }
  if (k >= st->max_iter) {
    st->status = DMP_NOT_CONVERGED;
    st->done = 1;
    return;
  }
  const double N = st->n_occ_d;
  st->step_kind = 0;
  if (st->method == DMP_METHOD_SP2) {
    const bool sq = fabs(t2 - N) <= fabs(2.0 * t1 - t2 - N);
    st->alpha = sq ? 0.0 : 2.0;
    st->b2 = sq ? 1.0 : -1.0;
    st->c = sq ? 1.0 : 0.0;
  } else {
    const double gamma = (N - (4.0 * t3 - 3.0 * t4)) / idem2;
    st->c = gamma;
    if (gamma > 6.0) {
      st->alpha = 2.0;
      st->b2 = -1.0;
    } else if (gamma < 0.0) {
      st->alpha = 0.0;
      st->b2 = 1.0;
    } else {
      st->step_kind = 1;
      st->zd = gamma;
      st->zx = 4.0 - 2.0 * gamma;
      st->zx2 = gamma - 3.0;
    }
  }
  st->iter = k + 1;
}

}  // namespace dmp
