// Chebyshev Fermi-operator expansion at finite electronic temperature (the
// finite-temperature method Sec. "Introduction" names: the Fermi Operator
// Expansion of Goedecker and Teter, Phys. Rev. B 51, 9455).
//
// P = f(H), f(e) = 1 / (1 + exp((e - mu) / kT)). H is scaled into [-1, 1] by a
// spectral enclosure [e_min, e_max] (a = centre, b = half-width, b = 1 for a
// point): H_s = (H - a I) / b. g(x) = f(a + b x) is expanded in M Chebyshev
// terms with coefficients from Gauss-Chebyshev quadrature on N = 2M nodes,
//   theta_j = pi (2j + 1) / (2N), x_j = cos(theta_j),
//   c_k = (2 / N) sum_j g(x_j) cos(k theta_j),
// and P = (c_0 / 2) I + sum_{k>=1} c_k T_k(H_s) with T_{k+1} = 2 H_s T_k - T_{k-1}.
// The products H_s T_k are formed by the product kernels of the library; this
// file holds the scalar set-up (enclosure, mu, coefficients) and the
// elementwise steps of the recurrence.
//
// Second evaluation of the same series (Paterson-Stockmeyer, after Liang et
// al., J. Chem. Phys. 119, 4117 (2003)): q = ceil(sqrt(M)) baby steps T_1 .. T_q
// are kept, the series is folded into sum_{m<r} T_m(y) B_m with y = T_q and
// B_m = sum_{j<q} w_{m,j} T_j (T_{qm+j} = 2 T_m(y) T_j - T_{qm-j}), and summed
// by Clenshaw's recurrence in y. Its kernels here: the next term of a
// recurrence, the weighted combination with the Clenshaw update, the
// Frobenius products <T_{qm}, T_j> and the trace assembly of canonical use,
// and the block folding of the coefficients.
//
// With a target n_occ, mu solves sum_k c_k(mu) tr T_k = n_occ. Writing
// w_j = t_0 / 2 + sum_{k>=1} t_k cos(k theta_j) (t_k = tr T_k from a first pass
// of the recurrence), the expansion's trace is (2 / N) sum_j g_mu(x_j) w_j, and
// mu is found by 100 bisection halvings of [e_min - 40 kT, e_max + 40 kT].
//
// cos(k theta_j) is evaluated as cospi(r / 2N) with r = k (2j + 1) mod 4N, an
// exact integer reduction, so large k lose no accuracy to the argument.
// Every sum runs in a fixed order: results are reproducible bit for bit.

#include <algorithm>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int kElemThreads = 256;
constexpr int kMaxRowBlocks = 4096;
constexpr int kReduceThreads = 1024;
constexpr double kMuBracketKT = 40.0;
constexpr int kMuHalvings = 100;

// Fermi-Dirac occupation without overflow.
__device__ __forceinline__ double fermi(double e, double mu, double kT) {
  const double z = (e - mu) / kT;
  if (z > 0.0) {
    const double ez = exp(-z);
    return ez / (1.0 + ez);
  }
  return 1.0 / (1.0 + exp(z));
}

// cos(k theta_j), theta_j = pi (2j + 1) / (2N)
__device__ __forceinline__ double cos_k_theta(int64_t k, int64_t j, int64_t N) {
  const int64_t r = (k * (2 * j + 1)) % (4 * N);
  return cospi(static_cast<double>(r) / static_cast<double>(2 * N));
}

__device__ __forceinline__ double node_x(int64_t j, int64_t N) {
  return cospi(static_cast<double>(2 * j + 1) / static_cast<double>(2 * N));
}

// Block-wide sum in a fixed tree (blockDim.x == kReduceThreads); every thread
// gets the total.
__device__ double block_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int o = kReduceThreads / 2; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  const double total = red[0];
  __syncthreads();
  return total;
}

// The enclosure that scales H: the caller's, else the Gershgorin bounds.
__global__ void foe_scale_kernel(const PurifyState* st, double e_min, double e_max, int use_given,
                                 FoeScalars* sc) {
  const double lo = use_given ? e_min : st->h_min;
  const double hi = use_given ? e_max : st->h_max;
  double b = 0.5 * (hi - lo);
  if (!(b > 0.0)) b = 1.0;
  sc->e_min = lo;
  sc->e_max = hi;
  sc->a = 0.5 * (hi + lo);
  sc->b = b;
  sc->nonfinite = st->nonfinite;
}

// w_j = t_0 / 2 + sum_{k=1}^{M-1} t_k cos(k theta_j), one thread per node.
__global__ void foe_weights_kernel(const double* __restrict__ traces, int M, double* __restrict__ w) {
  const int64_t N = 2 * static_cast<int64_t>(M);
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double acc = 0.5 * traces[0];
  for (int k = 1; k < M; ++k) acc += traces[k] * cos_k_theta(k, j, N);
  w[j] = acc;
}

// mu (bisection on the expansion's trace when `canonical`), then g(x_j) at
// that mu on every node. One CTA of kReduceThreads threads.
__global__ void __launch_bounds__(kReduceThreads)
foe_mu_kernel(FoeScalars* sc, double kT, double mu_given, double n_occ, int canonical, int M,
              const double* __restrict__ w, double* __restrict__ gx) {
  __shared__ double red[kReduceThreads];
  const int64_t N = 2 * static_cast<int64_t>(M);
  const double a = sc->a, b = sc->b;
  double mu = mu_given;
  if (canonical) {
    double lo = sc->e_min - kMuBracketKT * kT;
    double hi = sc->e_max + kMuBracketKT * kT;
    for (int it = 0; it < kMuHalvings; ++it) {
      const double mid = 0.5 * (lo + hi);
      double part = 0.0;
      for (int64_t j = threadIdx.x; j < N; j += kReduceThreads) part += fermi(a + b * node_x(j, N), mid, kT) * w[j];
      const double tr = (2.0 / static_cast<double>(N)) * block_sum(part, red);
      if (tr < n_occ) {
        lo = mid;
      } else {
        hi = mid;
      }
    }
    mu = 0.5 * (lo + hi);
  }
  for (int64_t j = threadIdx.x; j < N; j += kReduceThreads) gx[j] = fermi(a + b * node_x(j, N), mu, kT);
  if (threadIdx.x == 0) sc->mu = mu;
}

// c_k = (2 / N) sum_j g(x_j) cos(k theta_j), one thread per k.
__global__ void foe_coeff_kernel(const double* __restrict__ gx, int M, double* __restrict__ coeffs) {
  const int64_t N = 2 * static_cast<int64_t>(M);
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double acc = 0.0;
  for (int64_t j = 0; j < N; ++j) acc += gx[j] * cos_k_theta(k, j, N);
  coeffs[k] = (2.0 / static_cast<double>(N)) * acc;
}

// H_s = (H - a I) / b (upper triangle of H read, mirrored), T_0 = I, T_1 = H_s
// (each when its pointer is non-null), and, with coefficients,
// P = (c_0 / 2) I + c_1 H_s. Matrices of leading dimension n except H (ldh)
// and P (ldp).
__global__ void foe_init_kernel(const double* __restrict__ H, int64_t ldh, int64_t n, const FoeScalars* sc,
                                const double* __restrict__ coeffs, double* __restrict__ Hs, double* __restrict__ T0,
                                double* __restrict__ T1, double* __restrict__ P, int64_t ldp) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double a = sc->a, b = sc->b;
  const double c0h = coeffs ? 0.5 * coeffs[0] : 0.0;
  const double c1 = coeffs ? coeffs[1] : 0.0;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const double h = i <= j ? H[i * ldh + j] : H[j * ldh + i];
    const double d = i == j ? 1.0 : 0.0;
    const double hs = (h - (i == j ? a : 0.0)) / b;
    Hs[i * n + j] = hs;
    if (T0) T0[i * n + j] = d;
    if (T1) T1[i * n + j] = hs;
    if (coeffs) P[i * ldp + j] = c0h * d + c1 * hs;
  }
}

// T_{k+1} = 2 Y - T_{k-1} written over T_{k-1} (Y = H_s T_k), and, with P,
// P += c_{k+1} T_{k+1}.
__global__ void foe_step_kernel(const double* __restrict__ Y, double* __restrict__ Tprev, double* __restrict__ P,
                                int64_t ldp, const double* __restrict__ coeff, int64_t n) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double c = P ? *coeff : 0.0;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const double t = 2.0 * Y[i * n + j] - Tprev[i * n + j];
    Tprev[i * n + j] = t;
    if (P) P[i * ldp + j] += c * t;
  }
}

// out = sum_i A_ii in a fixed order (one CTA).
__global__ void __launch_bounds__(kReduceThreads)
foe_trace_kernel(const double* __restrict__ A, int64_t lda, int64_t n, double* __restrict__ out) {
  __shared__ double red[kReduceThreads];
  double part = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kReduceThreads) part += A[i * lda + i];
  const double total = block_sum(part, red);
  if (threadIdx.x == 0) *out = total;
}

// ---- Paterson-Stockmeyer evaluation (Liang et al., J. Chem. Phys. 119, 4117):
// baby steps T_1 .. T_q kept in q slots of n x n (T_0 = I implicit), y = T_q.

// Tout = 2 Y - Tprev, Tprev = I when null. Tout may be Tprev (in place).
__global__ void foe_next_kernel(const double* __restrict__ Y, const double* Tprev, double* Tout, int64_t n) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    const double prev = Tprev ? Tprev[i * n + j] : (i == j ? 1.0 : 0.0);
    Tout[i * n + j] = 2.0 * Y[i * n + j] - prev;
  }
}

// out = ((w_0 I + w_1 T_1 + ... + w_{nt-1} T_{nt-1}) + alpha Y) - Bm2, the Y and
// Bm2 terms only when their pointers are non-null. T_t lives at T + (t - 1) tstride.
// out (leading dimension ldo) may be Bm2 (in place).
__global__ void foe_combine_kernel(const double* __restrict__ T, int64_t tstride, int nt, const double* __restrict__ w,
                                   const double* __restrict__ Y, double alpha, const double* Bm2, double* out,
                                   int64_t ldo, int64_t n) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
    double v = i == j ? w[0] : 0.0;
    for (int t = 1; t < nt; ++t) v += w[t] * T[(t - 1) * tstride + i * n + j];
    if (Y) v += alpha * Y[i * n + j];
    if (Bm2) v -= Bm2[i * n + j];
    out[i * ldo + j] = v;
  }
}

// Frobenius products <G, T_t> for t = 1 .. nt - 1 (blockIdx.y = t - 1): per-block
// partial sums over the rows blockIdx.x, blockIdx.x + gridDim.x, ...
__global__ void __launch_bounds__(256)
foe_dots_kernel(const double* __restrict__ G, const double* __restrict__ T, int64_t tstride, int64_t n,
                double* __restrict__ partials) {
  __shared__ double red[8];
  const double* Tt = T + static_cast<int64_t>(blockIdx.y) * tstride;
  double acc = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) acc += G[i * n + j] * Tt[i * n + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    partials[static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

// out[t] = sum of the partial sums of product t, in a fixed order (one CTA per t).
__global__ void __launch_bounds__(kReduceThreads)
foe_dots_final_kernel(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  __shared__ double red[kReduceThreads];
  double part = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kReduceThreads)
    part += partials[static_cast<int64_t>(blockIdx.x) * nblocks + b];
  const double total = block_sum(part, red);
  if (threadIdx.x == 0) out[blockIdx.x] = total;
}

// tr T_k for every k < M from tr T_0 = n, the baby-step traces (k < q), the
// giant-step traces tr T_{qm} and the Frobenius products ip[m q + j] =
// <T_{qm}, T_j>: tr T_{qm+j} = 2 ip[m q + j] - tr T_{qm-j}. One thread.
__global__ void foe_ps_traces_kernel(double* traces, const double* __restrict__ ip, int q, int M, int64_t n) {
  traces[0] = static_cast<double>(n);
  for (int m = 1; q * m < M; ++m)
    for (int j = 1; j < q && q * m + j < M; ++j)
      traces[q * m + j] = 2.0 * ip[m * q + j] - traces[q * m - j];
}

// The weights w[m][j] of B_m = sum_{j<q} w[m][j] T_j, P = sum_{m<r} T_m(y) B_m:
// a_k = c_k (a_0 = c_0 / 2, zero past M), folded from the top block down
// (T_{qm+j} = 2 T_m(y) T_j - T_{qm-j}). One thread; a holds r q doubles.
__global__ void foe_fold_kernel(const double* __restrict__ coeffs, int M, int q, int r, double* __restrict__ a,
                                double* __restrict__ w) {
  for (int k = 0; k < r * q; ++k) a[k] = k < M ? coeffs[k] : 0.0;
  a[0] = 0.5 * coeffs[0];
  for (int m = r - 1; m > 0; --m) {
    w[m * q] = a[q * m];
    for (int j = 1; j < q; ++j) {
      const double d = a[q * m + j];
      w[m * q + j] = 2.0 * d;
      a[q * m - j] -= d;
    }
  }
  for (int j = 0; j < q; ++j) w[j] = a[j];
}

dim3 elem_grid(int64_t n) {
  return dim3(static_cast<unsigned>((n + kElemThreads - 1) / kElemThreads),
              static_cast<unsigned>(std::min<int64_t>(n, kMaxRowBlocks)));
}

}  // namespace

cudaError_t launch_foe_scale(const PurifyState* state, double e_min, double e_max, int use_given, FoeScalars* sc,
                             cudaStream_t st) {
  ProfScope prof(DMP_PROF_INIT, st);
  foe_scale_kernel<<<1, 1, 0, st>>>(state, e_min, e_max, use_given, sc);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_coefficients(FoeScalars* sc, double kT, double mu, double n_occ, const double* traces, int M,
                                    double* w, double* gx, double* coeffs, cudaStream_t st) {
  ProfScope prof(DMP_PROF_INIT, st);
  const int64_t N = 2 * static_cast<int64_t>(M);
  const int canonical = traces != nullptr;
  if (canonical) {
    foe_weights_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, st>>>(traces, M, w);
    count_launch();
  }
  foe_mu_kernel<<<1, kReduceThreads, 0, st>>>(sc, kT, mu, n_occ, canonical, M, w, gx);
  foe_coeff_kernel<<<static_cast<unsigned>((M + 127) / 128), 128, 0, st>>>(gx, M, coeffs);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_foe_init(const double* H, int64_t ldh, int64_t n, const FoeScalars* sc, const double* coeffs,
                            double* Hs, double* T0, double* T1, double* P, int64_t ldp, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  foe_init_kernel<<<elem_grid(n), kElemThreads, 0, st>>>(H, ldh, n, sc, coeffs, Hs, T0, T1, P, ldp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_step(const double* Y, double* Tprev, double* P, int64_t ldp, const double* coeff, int64_t n,
                            cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  foe_step_kernel<<<elem_grid(n), kElemThreads, 0, st>>>(Y, Tprev, P, ldp, coeff, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_next(const double* Y, const double* Tprev, double* Tout, int64_t n, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  foe_next_kernel<<<elem_grid(n), kElemThreads, 0, st>>>(Y, Tprev, Tout, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_combine(const double* T, int nt, const double* w, const double* Y, double alpha,
                               const double* Bm2, double* out, int64_t ldo, int64_t n, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  foe_combine_kernel<<<elem_grid(n), kElemThreads, 0, st>>>(T, n * n, nt, w, Y, alpha, Bm2, out, ldo, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_dots(const double* G, const double* T, int nt, int64_t n, double* partials, double* out,
                            cudaStream_t st) {
  if (nt < 2) return cudaSuccess;
  ProfScope prof(DMP_PROF_MEASURE, st);
  const dim3 grid(kFoeDotBlocks, static_cast<unsigned>(nt - 1));
  foe_dots_kernel<<<grid, 256, 0, st>>>(G, T, n * n, n, partials);
  foe_dots_final_kernel<<<static_cast<unsigned>(nt - 1), kReduceThreads, 0, st>>>(partials, kFoeDotBlocks, out);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_foe_ps_traces(double* traces, const double* ip, int q, int M, int64_t n, cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  foe_ps_traces_kernel<<<1, 1, 0, st>>>(traces, ip, q, M, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_fold(const double* coeffs, int M, int q, int r, double* a, double* w, cudaStream_t st) {
  ProfScope prof(DMP_PROF_INIT, st);
  foe_fold_kernel<<<1, 1, 0, st>>>(coeffs, M, q, r, a, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_foe_trace(const double* A, int64_t lda, int64_t n, double* out, cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  foe_trace_kernel<<<1, kReduceThreads, 0, st>>>(A, lda, n, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dmp
