/*
 * dmp.h -- density-matrix purification with Ozaki-scheme products on GB300.
 *
 * The problem (arXiv 2407.13299, Sec. "Density Matrix Purification"): given an
 * orthogonalised Hamiltonian H (n x n, symmetric; the Loewdin transform of Sec.
 * "Implementation Details" is done by the caller) and the number of occupied
 * orbitals n_occ, compute the density matrix P, the projector onto the n_occ
 * lowest eigenvectors of H (the spin-restricted K of the paper is 2P). P is
 * built by canonical purification (the Palser-Manolopoulos method the paper
 * cites), whose only heavy step is the dense product, and every product can be
 * emulated with the Ozaki error-free splitting scheme (Sec. "Ozaki Scheme",
 * Fig. 2): power-of-two row/column scaling, s digit slices per operand, exact
 * slice-pair products, FP64 recombination of the pairs with i + j <= s + 1.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major float64 in DEVICE memory owned by the caller,
 *     element (i, j) at ptr[i * ld + j], ld >= number of columns.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). All work is
 *     enqueued on it.
 *   - Workspace: every call that needs scratch takes a caller-allocated device
 *     buffer `ws` of `ws_bytes`, sized by the matching *_workspace_size call;
 *     the library allocates no device memory of its own (the one exception
 *     is the fixed array behind ozaki_gemm_noalloc).
 *   - Return value: 0 (DMP_OK) or a positive numerical status for purification
 *     (see below), or a negative error. No C++ exception crosses this ABI.
 *   - Thread safety: calls on different streams with different workspaces may
 *     run concurrently; a workspace must not be shared by calls in flight.
 */
#ifndef DMP_H
#define DMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- precision modes ------------------------------------------------------
 * DMP_FP64        every product in float64 (FP64 mma on the GPU).
 * DMP_OZAKI_INT8  Ozaki products with beta = 7 digit slices (|d| <= 127, the
 *                 int8 range): exact s32 accumulation of the level sums.
 * DMP_OZAKI_BF16  Ozaki products with beta = 8 digit slices rounded to nearest
 *                 (row exponent one larger, d_i = floor(y + 1/2), |d| <= 128,
 *                 integers bfloat16 holds exactly; digit products stay within
 *                 2^14 as for INT8 digits), tensor-core executor only. s in
 *                 [1, 9].
 * DMP_OZAKI_E4M3  Ozaki products with beta = 5 digit slices rounded to nearest
 *                 (the extraction of the original Ozaki scheme): the row
 *                 exponent is one larger (max_j |A_rj| < 2^(e_r - 1)) and
 *                 d_i = floor(y + 1/2) for y = 2^5 x, so |d| <= 16, integers
 *                 the FP8 format E4M3 holds exactly. Products run on the
 *                 tcgen05 kind::f8f6f4 tensor cores (fp32 accumulation in
 *                 tensor memory, exact while every partial sum stays below
 *                 2^24: a whole K of up to 65536 digits). s in [1, 12];
 *                 seven slices (34 bits below the row maximum) match five
 *                 INT8 slices (34). Tensor-core executor only.
 */
enum { DMP_FP64 = 0, DMP_OZAKI_INT8 = 1, DMP_OZAKI_BF16 = 2, DMP_OZAKI_E4M3 = 3 };

/* ---- executors for the slice-pair products ---------------------------------
 * DMP_EXEC_IMMA  int8 x int8 -> int32 warp-level tensor-core MMA.
 * DMP_EXEC_TC    digits carried in bfloat16 (E4M3 for DMP_OZAKI_E4M3) on the
 *                5th-generation tensor cores (tcgen05), fp32 accumulation in
 *                tensor memory, drained to exact integers every K chunk that
 *                keeps partial sums at most 2^24 in magnitude.
 * In the INT8 mode both give bit-identical level sums (the BF16 and E4M3
 * modes run on DMP_EXEC_TC only); DMP_EXEC_AUTO picks DMP_EXEC_TC.
 */
enum { DMP_EXEC_AUTO = 0, DMP_EXEC_IMMA = 1, DMP_EXEC_TC = 2 };

/* ---- return codes ------------------------------------------------------- */
enum {
  DMP_OK = 0,               /* converged: ||P^2 - P||_F < tol (or energy_tol met) */
  DMP_NOT_CONVERGED = 1,    /* max_iter reached                                    */
  DMP_STALLED = 2,          /* band energy rose on two steps by < 1e-2 (paper's halt rule) */
  DMP_C_OUT_OF_RANGE = 3,   /* tr(P - P^2) <= 0 or c outside [0, 1]: noise floor  */
  DMP_ERR_INVALID_ARG = -1, /* bad size, null pointer, ld < n, n_occ not in (0, n), s out of range */
  DMP_ERR_NONFINITE = -2,   /* NaN or Inf in an input or an iterate               */
  DMP_ERR_CUDA = -3,        /* a CUDA runtime call failed                          */
  DMP_ERR_TIMEOUT = -4,     /* a bounded device wait gave up                       */
  DMP_ERR_UNSUPPORTED = -5, /* mode/executor/size combination not available       */
  DMP_ERR_WORKSPACE = -6    /* ws_bytes (or tape_bytes) smaller than required      */
};

/* DMP_FLAG_BOUNDS_CONSTANT: dm_purify_backward treats the Gershgorin bounds
 * h_min, h_max of the initial guess as constants (no gradient through their
 * extreme rows). At convergence both choices agree to the convergence level,
 * because the converged projector does not depend on P_0. */
/* DMP_FLAG_FP32_STORAGE: every matrix the purification stores between
 * products (the initial guess, each P_k, each X^2, and for SP2/TRS4 the SP2
 * updates and the TRS4 factor Z) is rounded to the nearest FP32 value when it
 * is written, while the products, the recombination, the traces and the
 * coefficients stay in FP64: the storage experiment of Sec. "Mixed Precision
 * Purification", where matrices are held in FP32 and multiplied with FP64
 * accumulation. The buffers themselves stay FP64 (this reproduces the
 * precision of FP32 storage, not its memory saving). The refinement step
 * writes its result unrounded. Not offered with a tape, in the backward pass
 * or in the batched call (DMP_ERR_UNSUPPORTED). */
/* DMP_FLAG_BATCHED_STREAM: dm_purify_batched runs its iterations as ordinary
 * launches on the caller's stream, with a host read of the stopping rules
 * after every two iterations, instead of one CUDA-graph WHILE launch. The
 * kernels, their order and the results are the same; the host waits once per
 * two iterations. For profilers that cannot look inside conditional graph
 * nodes, and for per-phase times (dmp_profile_*), which are taken only outside
 * graphs. Ignored by the other calls. */
enum { DMP_FLAG_BOUNDS_CONSTANT = 1, DMP_FLAG_FP32_STORAGE = 2, DMP_FLAG_BATCHED_STREAM = 4 };

/*
 * Purification method (dmp_opts.method).
 * DMP_METHOD_PM    canonical purification (Palser-Manolopoulos; the default).
 * DMP_METHOD_TRS4  trace-resetting fourth-order purification, the recursion the
 *                  paper runs through NTPoly (Sec. "Implementation Details"):
 *                  X_0 = (h_max I - H)/(h_max - h_min); gamma = (n_occ - tr F)
 *                  / tr G with F = X^2 (4X - 3X^2), G = X^2 (I - X)^2; X' =
 *                  F + gamma G = X^2 Z, Z = gamma I + (4 - 2 gamma) X +
 *                  (gamma - 3) X^2, for gamma in [0, 6], else an SP2 step
 *                  (2X - X^2 above 6, X^2 below 0). Two products per step.
 * DMP_METHOD_SP2   second-order spectral projection: X' = X^2 or 2X - X^2,
 *                  whichever brings tr X' closer to n_occ. One product per step.
 * For TRS4 and SP2, tr G is taken as ||X^2 - X||_F^2 and the stopping rules
 * are: ||X^2 - X||_F < tol (DMP_OK); k >= 2, the value two steps earlier
 * below 1 and not above the current one (the rounding floor,
 * DMP_C_OUT_OF_RANGE); k == max_iter (DMP_NOT_CONVERGED). No energy rules.
 * They take no tape and are not offered in the batched call.
 */
enum { DMP_METHOD_PM = 0, DMP_METHOD_TRS4 = 1, DMP_METHOD_SP2 = 2 };

/* Options. Zero-initialise and set what you need; zeros select defaults. */
typedef struct {
  int32_t mode;             /* DMP_FP64 / DMP_OZAKI_INT8 / DMP_OZAKI_BF16 / _E4M3   */
  int32_t slices;           /* s in [1, 10] (beta 7), [1, 9] (beta 8) or [1, 12]
                               (E4M3); 0 -> 7                                        */
  int32_t executor;         /* DMP_EXEC_*                                            */
  int32_t max_iter;         /* 0 -> 100 (the paper's cap)                            */
  int32_t checkpoint_every; /* forward iterates kept every k steps for the adjoint; 0 -> 8 */
  int32_t flags;            /* DMP_FLAG_* bits                                       */
  double tol;               /* ||P^2 - P||_F threshold; 0 -> 1e-10                   */
  double energy_tol;        /* optional |change of Tr(HK)| threshold; 0 = off        */
  int32_t refine_slices;    /* refinement after the loop (see dm_purify): 0 off,
                               -1 FP64 products, s_r > 0 Ozaki products of s_r slices */
  int32_t method;           /* DMP_METHOD_* (0: canonical purification)              */
  int32_t late_slices;      /* late-slice schedule (see dm_purify): 0 off, else the
                               slice count of every pass after an iterate with
                               ||P^2 - P||_F < late_idem                              */
  double late_idem;         /* threshold of the late-slice schedule                  */
} dmp_opts;

/* Per-run report, filled when the host pointer is non-NULL (the call then
 * synchronises the stream before returning). */
typedef struct {
  int32_t status;      /* DMP_OK .. DMP_C_OUT_OF_RANGE, or a negative error     */
  int32_t iters;       /* purification updates applied                         */
  int32_t slices_used; /* s (0 in FP64 mode)                                     */
  int32_t executor_used;
  double energy;       /* tr(P H)                                                */
  double band_energy;  /* Tr(H K) = 2 tr(P H), the paper's energy                */
  double idem;         /* ||P^2 - P||_F of the returned P                        */
  double trace;        /* tr(P)                                                  */
  double c_last;       /* last coefficient: c (canonical), gamma (TRS4), 1 or 0 for a
                          squaring or a 2X - X^2 step (SP2)                       */
  double h_min, h_max; /* Gershgorin bounds used for the initial guess          */
  double energy_unrefined; /* tr(P H) before the refinement step (= energy if none) */
  int32_t refined;     /* 1 if the refinement step was applied                   */
  int32_t late_iters;  /* passes (P^2 products) formed with late_slices slices     */
} dmp_info;

/* Bytes of workspace dm_purify needs for this n and these options. */
int dmp_workspace_size(int64_t n, const dmp_opts* opts, size_t* bytes);

/* Bytes of the adjoint tape dm_purify writes when given one (checkpoints every
 * opts->checkpoint_every iterates plus per-step scalars). */
int dmp_tape_size(int64_t n, const dmp_opts* opts, size_t* bytes);

/*
 * dm_purify: canonical purification of H (Sec. "Density Matrix Purification";
 * initial guess from the Gershgorin bounds, coefficient
 * c = tr(P^2 - P^3) / tr(P - P^2), update
 *   c >= 1/2: P' = ((1 + c) P^2 - P^3) / c,
 *   c <  1/2: P' = ((1 - 2c) P + (1 + c) P^2 - P^3) / (1 - c)),
 * every product in opts->mode. Stopping rules, tested in this order on each
 * iterate P_k: ||P_k^2 - P_k||_F < tol (DMP_OK); the paper's energy halt rule
 * (DMP_STALLED); |change of band energy| < energy_tol if set (DMP_OK);
 * k == max_iter (DMP_NOT_CONVERGED); tr(P - P^2) <= 0 or c outside [0, 1]
 * (DMP_C_OUT_OF_RANGE). The returned P is that P_k, or, with
 * opts->refine_slices != 0 and a status >= 0, its refinement: one McWeeny step
 * P' = 3 P_k^2 - 2 P_k^3 in full precision (Sec. "Precision Requirements
 * Sweep": the paper's mixed-precision recommendation when the energy matters),
 * with FP64 products (refine_slices = -1) or Ozaki products of refine_slices
 * slices (9 reaches FP64 accuracy; the level-sum limit below applies to it).
 * info->energy then describes P' and info->energy_unrefined P_k; info->idem
 * stays that of P_k. Refinement with a tape is DMP_ERR_UNSUPPORTED.
 * Late-slice schedule (an option of this library; the paper weighs adjusting
 * the precision across iterations in Sec. "Precision Requirements Sweep"):
 * with opts->late_slices = s_l > 0, once an iterate has ||P_k^2 - P_k||_F <
 * opts->late_idem, every later pass forms its products with s_l slices (the
 * switch applies from pass k + 1 and is never undone; info->late_iters counts
 * those passes). A product error disturbs the occupied subspace in proportion
 * to the error over the gap between the iterate's occupied and virtual
 * eigenvalues, and that gap grows geometrically along the loop, so late
 * passes tolerate fewer slices, the more so with the refinement step, which
 * repairs the eigenvalues. Canonical purification only; not with a tape.
 *   H      n x n, leading dimension ldh. Only the upper triangle is read; the
 *          lower triangle is taken as its mirror.
 *   P      n x n output, leading dimension ldp (may not alias H).
 *   info   host pointer or NULL (then nothing is reported).
 *          The call synchronises `stream` once per iteration to read the
 *          device-side stopping decision, and before it returns.
 *   tape   NULL, or a device buffer of dmp_tape_size bytes that receives what
 *          dm_purify_backward needs.
 * Returns the status (>= 0) or a negative error.
 */
int dm_purify(const double* H, int64_t n, int64_t ldh, int64_t n_occ, const dmp_opts* opts,
              double* P, int64_t ldp, dmp_info* info, void* ws, size_t ws_bytes,
              void* tape, size_t tape_bytes, void* stream);

/* Bytes of device workspace dm_purify_host needs for this n and these
 * options: room for device copies of H and P (2 n^2 doubles) followed by
 * dm_purify's workspace. */
int dmp_host_workspace_size(int64_t n, const dmp_opts* opts, size_t* bytes);

/*
 * dm_purify_host: dm_purify with H and P in HOST memory -- the problem as Sec.
 * "Density Matrix Purification" states it, Hamiltonian in and density matrix
 * out, with both transfers inside the library's boundary.
 *   H_host  n x n row-major float64 in host memory, leading dimension ldh
 *           (upper triangle read, as for dm_purify).
 *   P_host  n x n host output, leading dimension ldp (may not alias H_host).
 *   ws      DEVICE workspace of dmp_host_workspace_size bytes: H is copied to
 *           its front with one cudaMemcpy2DAsync on `stream`, dm_purify runs
 *           on that copy with the rest of the workspace, and P is copied back
 *           with one cudaMemcpy2DAsync on `stream`.
 * The call synchronises `stream` before it returns, so P_host holds the result
 * (and H_host may be reused) on return. Page-locked host buffers make both
 * copies DMA transfers at full link speed; pageable ones work but the driver
 * stages them. P_host is written only when the status is >= 0. Options,
 * statuses and errors are those of dm_purify; there is no tape (the adjoint
 * needs the device-resident dm_purify).
 */
int dm_purify_host(const double* H_host, int64_t n, int64_t ldh, int64_t n_occ, const dmp_opts* opts,
                   double* P_host, int64_t ldp, dmp_info* info, void* ws, size_t ws_bytes, void* stream);

/* Bytes of workspace ozaki_gemm needs. */
int ozaki_gemm_workspace_size(int64_t m, int64_t n, int64_t k, int32_t mode, int32_t slices,
                              int32_t executor, size_t* bytes);

/*
 * ozaki_gemm: C = A B, m x k times k x n, through the Ozaki scheme
 * (Sec. "Ozaki Scheme"): A scaled per row and B per column by powers of two,
 * split into `slices` digit planes of beta bits (mode DMP_OZAKI_INT8: beta 7;
 * DMP_OZAKI_BF16: beta 8 and DMP_OZAKI_E4M3: beta 5, both nearest digits), level sums
 * S_L = sum_{i+j=L} A_i B_j formed exactly for L = 2..s+1, and
 * C = 2^(e_r+f_c) * sum_L S_L 2^(-beta L) in float64: groups of up to four
 * consecutive levels (beta 7 and 5; three for beta 8) are first combined
 * exactly in 64-bit integers, then the groups are added in float64 from the
 * L = s+1 end to L = 2. With at most two groups (s <= 8 for beta 7 and 5,
 * s <= 6 for beta 8) this is the correctly rounded value of the exact sum of
 * the kept pairs. The result is bit-for-bit the same for every executor. mode DMP_FP64
 * computes a plain float64 product instead.
 * A row of A or column of B holding NaN/Inf gives a NaN row/column of C.
 * Limits: s * k * dmax^2 < 2^31 (exact s32 level sums; dmax = 127 for INT8,
 * 128 for BF16, 16 for E4M3).
 */
int ozaki_gemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
               int64_t ldb, double* C, int64_t ldc, int32_t mode, int32_t slices, int32_t executor,
               void* ws, size_t ws_bytes, void* stream);

/*
 * ozaki_gemm_noalloc: ozaki_gemm without a workspace argument. (The paper has
 * no counterpart; this is a convenience of this library.)
 *
 * Some callers cannot supply device scratch memory: a C or Fortran host code
 * that has no device allocator of its own to size and keep a buffer alive, or
 * a caller in the middle of its own GPU pipeline that must not allocate
 * because a device allocation can synchronise the device and stall its other
 * streams. This entry point serves them. It computes exactly what ozaki_gemm
 * computes (same kernels, same bits), with all scratch taken from one fixed
 * 128 MiB array in device memory that the library defines. The call makes no
 * allocation of its own (no cudaMalloc/cudaFree, no allocating library call).
 *   - The array belongs to the library: every GPU that loads it keeps the
 *     128 MiB until the process exits.
 *   - Every call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress with the caller's device current) instead of
 *     keeping it, so a context created anew after cudaDeviceReset gets the
 *     array's new address. The first call on a device may load the library's
 *     device code; make it before any stream capture.
 *   - All calls share the one array, so calls that overlap on the GPU (on
 *     different streams, or from several threads) race and give undefined
 *     results. Serialise them.
 *   - Problems whose scratch (as ozaki_gemm_workspace_size reports it) exceeds
 *     128 MiB are rejected with DMP_ERR_WORKSPACE before any work is enqueued.
 *     At s = 7 square problems fit up to m = n = k = 1056 in the INT8 and BF16
 *     modes on the tcgen05 executor (two-byte digits and an 80 MiB partial-sum
 *     area), 1440 in the E4M3 mode and 2432 on the int8 mma executor.
 *     DMP_FP64 needs no scratch.
 * Arguments and the other return codes are those of ozaki_gemm.
 */
int ozaki_gemm_noalloc(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                       const double* B, int64_t ldb, double* C, int64_t ldc, int32_t mode,
                       int32_t slices, int32_t executor, void* stream);

/*
 * ozaki_level_sums: the exact integer slice-pair products of ozaki_gemm,
 * S[L-2][i][j] = (sum_{a+b=L} A_a B_b)[i][j] as int32, L = 2..s+1, written to
 * S (s x m x n, row-major, leading dimension n). Exposed so that the integer
 * part of the scheme can be compared bit for bit. Same workspace as ozaki_gemm.
 */
int ozaki_level_sums(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                     const double* B, int64_t ldb, int32_t* S, int32_t mode, int32_t slices,
                     int32_t executor, void* ws, size_t ws_bytes, void* stream);

/*
 * ozaki_split: the row scaling and digit planes of A (m x k), the first step
 * of the scheme, exactly as the product kernels consume them. exps[m] receives
 * e_r (max_j |A_rj| < 2^e_r, or < 2^(e_r - 1) for the nearest digits of
 * DMP_OZAKI_BF16 and DMP_OZAKI_E4M3; 0 for a
 * zero row; INT32_MAX for a row holding NaN or Inf, whose products are then
 * NaN). digits receives s planes of m x k (plane-major, leading dimension k)
 * of the digits: int8 for executor DMP_EXEC_IMMA, bfloat16 bit patterns for
 * DMP_EXEC_TC (truncated 7-bit digits, or nearest 8-bit ones for
 * DMP_OZAKI_BF16); for DMP_OZAKI_E4M3
 * the nearest digits (|d| <= 16) as E4M3 bytes (sign bit 7, exponent bits
 * 3..6 with bias 7, fraction bits 0..2). Workspace as for
 * ozaki_gemm(m, 1, k, ...).
 */
int ozaki_split(int64_t m, int64_t k, const double* A, int64_t lda, int32_t mode, int32_t slices,
                int32_t executor, int32_t* exps, void* digits, void* ws, size_t ws_bytes,
                void* stream);

/* Workspace for the batched call below. */
int dmp_batched_workspace_size(int32_t batch, const int64_t* n, const dmp_opts* opts, size_t* bytes);

/*
 * dm_purify_batched: purify `batch` independent Hamiltonians of possibly
 * different sizes with the same options. Each member is the canonical
 * purification of Sec. "Density Matrix Purification" (the method of dm_purify,
 * with the Ozaki products of Sec. "Ozaki Scheme"); the paper purifies one
 * system at a time, and grouping many small ones into shared launches is this
 * library's scheduling, which changes no member's arithmetic. H, P, n and n_occ are HOST arrays of
 * length `batch`; H[b] and P[b] are device pointers (n[b] x n[b], leading
 * dimension n[b]). infos (host, length batch, nullable) receives one report per
 * matrix. Each matrix stops on its own rule; the call returns DMP_OK when all
 * converged, else the largest status seen. Modes DMP_OZAKI_INT8, DMP_OZAKI_BF16
 * and DMP_OZAKI_E4M3 (DMP_FP64 gives DMP_ERR_UNSUPPORTED).
 * opts->refine_slices = r > 0 adds the refinement step of dm_purify (one
 * McWeeny step P' = 3 P^2 - 2 P^3 with r-slice products, Sec. "Precision
 * Requirements Sweep") to every member that ended without an error, after the
 * whole batch has stopped; its report then holds the refined energy
 * (refined = 1). FP64 refinement products (r < 0), FP32 storage and the
 * late-slice schedule are not offered here (DMP_ERR_UNSUPPORTED). With
 * opts->slices = 0 the slice-count tuner compares refined energies.
 */
int dm_purify_batched(int32_t batch, const double* const* H, const int64_t* n,
                      const int64_t* n_occ, double* const* P, const dmp_opts* opts,
                      dmp_info* infos, void* ws, size_t ws_bytes, void* stream);

/* Workspace for the backward call below. */
int dmp_backward_workspace_size(int64_t n, const dmp_opts* opts, size_t* bytes);

/*
 * dm_purify_backward: reverse mode through the purification that dm_purify
 * ran with `tape` and the same options, giving dL/dH for a loss L(P) from
 * G = dL/dP (n x n, leading dimension n). The forward is the canonical
 * purification of Sec. "Density Matrix Purification" (the update of the cited
 * Palser-Manolopoulos method, products by the Ozaki scheme); the paper does
 * not differentiate it, and this is the exact adjoint of that iteration. Each step k is differentiated with
 * its branch and the iteration count frozen and with the dependence of the
 * coefficient c_k on P_k kept:
 *   dL/dP_k = alpha G + b2 (G P + P G) + b3 (G P^2 + P G P + P^2 G)
 *             + <G, alpha' P + b2' P^2 + b3' P^3> dc/dP,
 *   dc/dP = ((2P - 3P^2) tr(P - P^2) - tr(P^2 - P^3)(I - 2P)) / tr(P - P^2)^2,
 * (alpha, b2, b3) the weights of the branch c selected and ' their derivatives
 * in c), then through the initial guess: the direct term -(lambda/n) G_0, the
 * trace term of mu = tr(H)/n and lambda through its active branch and the
 * Gershgorin extreme rows (unless opts->flags has DMP_FLAG_BOUNDS_CONSTANT).
 * The iterates are recomputed from the tape's checkpoints segment by segment
 * (bit-identical to the forward's); products run in the forward's mode.
 *   H     the forward's H, leading dimension n.
 *   dLdH  n x n, leading dimension n: the gradient for symmetric H, i.e. the
 *         symmetric part of the gradient with respect to H as a general
 *         matrix. A perturbation of H_ij and H_ji by h changes L by
 *         2 h dLdH[i][j] (i != j); of H_ii by h, by h dLdH[i][i].
 * The call synchronises `stream` once per checkpoint segment and on return.
 */
int dm_purify_backward(const double* H, int64_t n, int64_t n_occ, const dmp_opts* opts,
                       const void* tape, size_t tape_bytes, const double* dLdP, double* dLdH,
                       void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- finite temperature
 * Fermi-operator expansion: the finite-temperature method the paper names for
 * metallic systems, where purification does not apply (Sec. "Introduction":
 * the Fermi Operator Expansion of Goedecker and Teter, Phys. Rev. B 51, 9455;
 * the paper's own experiments with it are in its Supplementary Information).
 */
enum { DMP_FOE_MAX_TERMS = 16384 };

/* Evaluation of the series (dmp_foe_params.scheme).
 * DMP_FOE_RECURRENCE            the three-term recurrence: M - 2 products per pass.
 * DMP_FOE_PATERSON_STOCKMEYER   the Paterson-Stockmeyer evaluation of Liang et al.
 *                               (J. Chem. Phys. 119, 4117 (2003)): q = ceil(sqrt(M))
 *                               baby steps T_1 .. T_q kept, the series folded into
 *                               sum_{m<r} T_m(y) B_m (y = T_q, r = ceil(M/q), B_m a
 *                               combination of T_0 .. T_{q-1}) and summed by
 *                               Clenshaw's recurrence in y: (q - 1) + (r - 1)
 *                               products, plus r - 2 giant steps T_m(y) whose traces
 *                               (tr T_{qm+j} = 2 <T_{qm}, T_j>_F - tr T_{qm-j})
 *                               replace the first pass when mu is solved. Holds q
 *                               n x n matrices more than the recurrence. */
enum { DMP_FOE_RECURRENCE = 0, DMP_FOE_PATERSON_STOCKMEYER = 1 };

/* Parameters of dm_foe. */
typedef struct {
  double kT;           /* electronic temperature, in the energy units of H; > 0       */
  double mu;           /* chemical potential, used when n_occ == 0                    */
  int64_t n_occ;       /* 0: mu as given; 0 < n_occ < n: mu is solved so that
                          tr(P) = n_occ (the recurrence then runs twice)              */
  int32_t n_terms;     /* Chebyshev terms M in [2, DMP_FOE_MAX_TERMS]                 */
  int32_t scheme;      /* DMP_FOE_RECURRENCE (0) or DMP_FOE_PATERSON_STOCKMEYER       */
  double e_min, e_max; /* enclosure of the spectrum of H that scales it into [-1, 1];
                          e_min >= e_max (e.g. both 0) selects the Gershgorin bounds  */
} dmp_foe_params;

/* Report of dm_foe, filled when the host pointer is non-NULL. */
typedef struct {
  int32_t status;      /* DMP_OK or a negative error                                */
  int32_t n_terms;     /* M                                                          */
  int32_t products;    /* matrix products formed (see the schemes above)             */
  int32_t slices_used; /* s (0 in FP64 mode)                                         */
  double mu;           /* chemical potential of the result                           */
  double trace;        /* tr(P)                                                      */
  double energy;       /* tr(P H)                                                    */
  double band_energy;  /* 2 tr(P H)                                                  */
  double e_min, e_max; /* the enclosure that scaled H                                */
  double tail;         /* |c_{M-2}| + |c_{M-1}|: size of the last two coefficients, a
                          guide to the truncation error of the expansion              */
} dmp_foe_info;

/* Bytes of workspace dm_foe needs for this n, these parameters (only n_terms
 * and scheme matter) and these options. */
int dm_foe_workspace_size(int64_t n, const dmp_foe_params* params, const dmp_opts* opts, size_t* bytes);

/*
 * dm_foe: P = f(H), f(e) = 1 / (1 + exp((e - mu) / kT)) (occupations in [0, 1];
 * the paper's K = 2P), by a Chebyshev expansion whose matrix products are
 * formed in opts->mode:
 *   a = (e_max + e_min) / 2, b = (e_max - e_min) / 2 (b = 1 if the enclosure
 *   is a point), H_s = (H - a I) / b;
 *   c_k = (2 / N) sum_j f(a + b x_j) cos(k theta_j), k < M, on the N = 2M
 *   Gauss-Chebyshev nodes theta_j = pi (j + 1/2) / N, x_j = cos(theta_j);
 *   P = (c_0 / 2) I + sum_{k=1}^{M-1} c_k T_k(H_s), T_0 = I, T_1 = H_s,
 *   T_{k+1} = 2 H_s T_k - T_{k-1}, or the Paterson-Stockmeyer scheme above;
 *   every product is symmetric (its upper triangle is formed and mirrored) and
 *   H_s (and y = T_q) is split once per call.
 * With params->n_occ > 0, the traces tr T_k come first (a first pass of the
 * recurrence, or the giant steps of the Paterson-Stockmeyer scheme) and mu
 * solves sum_k c_k(mu) tr T_k = n_occ by 100 bisection halvings of
 * [e_min - 40 kT, e_max + 40 kT]; then P is formed.
 * The truncation error falls roughly like exp(-M pi kT / b): M must grow with
 * b / kT, so a tight enclosure matters (Gershgorin bounds of a dense H can be
 * several times wider than its spectrum). An enclosure that misses part of the
 * spectrum makes the series diverge there.
 * Options used: mode, slices, executor; refine_slices, late_slices, method and
 * DMP_FLAG_FP32_STORAGE must be zero/unset (else DMP_ERR_UNSUPPORTED).
 *   H      n x n, leading dimension ldh; only the upper triangle is read.
 *   P      n x n output, leading dimension ldp (may not alias H or ws).
 *   ws     device workspace of dm_foe_workspace_size bytes.
 * Errors: DMP_ERR_INVALID_ARG (null pointer, n < 2, ld < n, kT not positive and
 * finite, mu not finite with n_occ == 0, n_occ outside [0, n), M outside
 * [2, DMP_FOE_MAX_TERMS], an unknown scheme, a non-finite enclosure),
 * DMP_ERR_NONFINITE (H holds a
 * NaN/Inf), DMP_ERR_UNSUPPORTED (options above, or the level-sum limit of
 * ozaki_gemm for k = n), DMP_ERR_WORKSPACE, DMP_ERR_TIMEOUT, DMP_ERR_CUDA.
 * The call synchronises `stream` after the Gershgorin pass and before it returns.
 */
int dm_foe(const double* H, int64_t n, int64_t ldh, const dmp_foe_params* params, const dmp_opts* opts,
           double* P, int64_t ldp, dmp_foe_info* info, void* ws, size_t ws_bytes, void* stream);

/* Kernel timing. While enabled, every kernel launch of the library is
 * bracketed by two CUDA events recorded on the launching stream, tagged with
 * its class: DMP_PROF_PRODUCT (slice-pair / FP64 product kernels), DMP_PROF_SPLIT
 * (scaling and digit split), DMP_PROF_MEASURE (traces, norms, stopping rules),
 * DMP_PROF_INIT (Gershgorin bounds and initial guess), DMP_PROF_OTHER.
 * dmp_profile_read synchronises the recorded events and returns the summed
 * device time (ms) and the launch count of one class. Host-side, process-wide,
 * guarded by a mutex. */
enum { DMP_PROF_PRODUCT = 0, DMP_PROF_SPLIT = 1, DMP_PROF_MEASURE = 2, DMP_PROF_INIT = 3, DMP_PROF_OTHER = 4 };
int dmp_profile_enable(int on);
int dmp_profile_reset(void);
int dmp_profile_read(int32_t kind, double* total_ms, long long* launches);

/* Name of a return code. */
const char* dmp_status_str(int code);

/* Number of kernels this library has launched since load (all threads). */
long long dmp_launch_count(void);

/* Library version string. */
const char* dmp_version(void);

/* Whether DMP_EXEC_TC products with beta = 7 run on CTA pairs: clusters of two
 * CTAs on neighbouring SMs that compute 256 x 256 output tiles with the 2-SM
 * tensor-core MMA (each SM stages its own 128 rows of A and half of B). On by
 * default; off runs one CTA per 128 x 256 tile. Both give bit-identical
 * results (the same exact integer level sums). Process-wide, read at each
 * launch; returns the previous setting. A performance knob with no
 * counterpart in the paper. */
int dmp_set_tc_pairing(int enable);

/* Whether single-matrix DMP_EXEC_TC products split their output tiles when
 * they fill at most half a wave of the persistent kernel (one CTA, or CTA
 * pair, per SM): the tiles are then cut into units of one exact fp32 chunk and
 * shared out evenly over every CTA, so the idle part of the GPU works too
 * (n <= 2048 in the purification on GB300: 25-40 % less product time). The
 * partial level sums are
 * integers added at L2, so any split gives the same exact sums and the result
 * is bit-for-bit that of whole tiles. Used by dm_purify, dm_purify_backward and
 * dm_foe (their workspaces include the room it needs), with at most two level
 * groups (s <= 8 for beta 7 and 5, s <= 6 for beta 8); ozaki_gemm runs whole
 * tiles. On by default. Process-wide, read at each launch; returns the
 * previous setting. A performance knob with no counterpart in the paper. */
int dmp_set_tc_split_tiles(int enable);

/* Tile shape of dm_purify_batched's grouped product: 0 (the default) lets the
 * library's autotuner pick it by timing the batch's first product; 128 or 256
 * force single-CTA tiles of 128 x 128 or 128 x 256, 512 forces CTA pairs on
 * 256 x 256 tiles (E4M3 digits: 256 or 512 only). For reproducible runs and for
 * profilers, whose replays would distort the tuner's timing. Process-wide, read
 * at each call; returns the previous setting, or DMP_ERR_INVALID_ARG (setting
 * unchanged) for another value. dm_purify_batched returns DMP_ERR_UNSUPPORTED
 * when the forced shape is not available for its mode or on this GPU. A
 * performance knob with no counterpart in the paper. */
int dmp_set_batched_tile(int tile);

/* Test hook for the bounded device waits (no counterpart in the paper). The
 * next tcgen05 product launch of the process (from any single-matrix entry
 * point, on any stream) is started with every wait bounded by wait_limit_us
 * microseconds instead of the
 * normal 5 s, and each of its CTAs withholds the operand copies of its first
 * pipeline stage: that stage's barrier never completes, so the MMA issuer's
 * wait on it runs out. The kernel then takes its abort path -- it raises the
 * call's error flag, waits (bounded) for the copies it did issue, frees its
 * tensor memory and returns -- and the call reports DMP_ERR_TIMEOUT. Nothing
 * faults and nothing is left running; the next call is unaffected. One-shot:
 * the setting is consumed by that launch. 0 cancels a pending request; a
 * negative limit is DMP_ERR_INVALID_ARG. Launches being captured into a CUDA
 * graph, the grouped launches of dm_purify_batched, the int8 mma executor and
 * the FP64 products do not take it. */
int dmp_test_stall_next_product(int32_t wait_limit_us);

#ifdef __cplusplus
}
#endif

#endif /* DMP_H */
