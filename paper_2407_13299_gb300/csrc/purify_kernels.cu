// Initial guess, per-iterate measures and the stopping rules of canonical
// purification (the Palser-Manolopoulos method cited in Sec. "Introduction";
// halt rules of Sec. "Implementation Details"). All in float64.
//
// Symmetry: only the upper triangle of H is read (element (i, j) is taken as
// H[min(i,j)][max(i,j)]), so P_0 and every iterate are exactly symmetric. The
// measures of an iterate use that symmetry too: each reduction reads the upper
// triangle and doubles the strictly-upper part.
//
// Reductions are deterministic: fixed grid, fixed per-thread order, fixed tree.
//
// Also here: the elementwise SP2 step and TRS4 factor, the refinement weights
// and energy, and the FP32-storage rounding of every matrix these kernels
// store (stored_value, DMP_FLAG_FP32_STORAGE).

#include <algorithm>

#include "dmp_internal.cuh"

namespace dmp {

namespace {

constexpr int kRowThreads = 256;
constexpr int kColChunks = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Strictly-upper row sums U_i = sum_{j>i} |H_ij| and the diagonal, one CTA per row.
__global__ void __launch_bounds__(kRowThreads)
gersh_rows_kernel(const double* __restrict__ H, int64_t n, int64_t ldh, double* __restrict__ U,
                  double* __restrict__ D, int* __restrict__ flag) {
  const int64_t i = blockIdx.x;
  __shared__ double red[kRowThreads / 32];
  double sacc = 0.0;
  bool bad = false;
  const double* row = H + i * ldh;
  for (int64_t j = i + 1 + threadIdx.x; j < n; j += kRowThreads) {
    const double v = row[j];
    bad |= !isfinite(v);
    sacc += fabs(v);
  }
  sacc = warp_sum(sacc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sacc;
  if (bad) atomicExch(flag, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRowThreads / 32; ++w) t += red[w];
    U[i] = t;
    const double d = row[i];
    if (!isfinite(d)) atomicExch(flag, 1);
    D[i] = d;
  }
}

// Column partial sums of the strict upper triangle: Cp[chunk][c] = sum over rows
// r < c of the chunk of |H_rc|. Threads own columns, so reads are coalesced.
__global__ void gersh_cols_kernel(const double* __restrict__ H, int64_t n, int64_t ldh,
                                  double* __restrict__ Cp) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y;
  if (c >= n) return;
  const int64_t rows_per = (n + kColChunks - 1) / kColChunks;
  const int64_t r0 = chunk * rows_per;
  const int64_t r1 = min(r0 + rows_per, c);
  double sacc = 0.0;
  for (int64_t r = r0; r < r1; ++r) sacc += fabs(H[r * ldh + c]);
  Cp[static_cast<int64_t>(chunk) * n + c] = sacc;
}

// Bounds, mu, lambda -> state. One CTA.
__global__ void __launch_bounds__(1024)
gersh_final_kernel(int64_t n, int64_t n_occ, const double* __restrict__ U, const double* __restrict__ D,
                   const double* __restrict__ Cp, PurifyState* st, const int* flag) {
  __shared__ double s_lo[1024], s_hi[1024], s_tr[1024];
  __shared__ int s_ilo[1024], s_ihi[1024];
  const int t = threadIdx.x;
  double lo = 1.0 / 0.0, hi = -1.0 / 0.0, tr = 0.0;
  int ilo = 0x7fffffff, ihi = 0x7fffffff;
  for (int64_t i = t; i < n; i += blockDim.x) {
    double rad = U[i];
    for (int ch = 0; ch < kColChunks; ++ch) rad += Cp[static_cast<int64_t>(ch) * n + i];
    const double l = D[i] - rad, h = D[i] + rad;
    if (l < lo) { lo = l; ilo = static_cast<int>(i); }
    if (h > hi) { hi = h; ihi = static_cast<int>(i); }
    tr += D[i];
  }
  s_lo[t] = lo; s_hi[t] = hi; s_tr[t] = tr; s_ilo[t] = ilo; s_ihi[t] = ihi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) {
      // keep the first index on ties
      if (s_lo[t + o] < s_lo[t] || (s_lo[t + o] == s_lo[t] && s_ilo[t + o] < s_ilo[t])) {
        s_lo[t] = s_lo[t + o];
        s_ilo[t] = s_ilo[t + o];
      }
      if (s_hi[t + o] > s_hi[t] || (s_hi[t + o] == s_hi[t] && s_ihi[t + o] < s_ihi[t])) {
        s_hi[t] = s_hi[t + o];
        s_ihi[t] = s_ihi[t + o];
      }
      s_tr[t] += s_tr[t + o];
    }
    __syncthreads();
  }
  if (t == 0) {
    const double dn = static_cast<double>(n);
    const double mu = s_tr[0] / dn;
    st->h_min = s_lo[0];
    st->h_max = s_hi[0];
    st->row_min = s_ilo[0];
    st->row_max = s_ihi[0];
    st->mu = mu;
    if (*flag) {
      st->nonfinite = 1;
      st->status = DMP_ERR_NONFINITE;
      st->done = 1;
      st->lam = 0.0;
      return;
    }
    if (!(s_hi[0] > mu && mu > s_lo[0])) {  // H is a multiple of the identity
      st->status = DMP_ERR_INVALID_ARG;
      st->done = 1;
      st->lam = 0.0;
      return;
    }
    st->n_occ_d = static_cast<double>(n_occ);
    const double lam1 = static_cast<double>(n_occ) / (s_hi[0] - mu);
    const double lam2 = static_cast<double>(n - n_occ) / (mu - s_lo[0]);
    st->lam_branch = lam1 <= lam2 ? 1 : 2;
    st->lam = lam1 <= lam2 ? lam1 : lam2;
  }
}

// P0 = (lambda/n)(mu I - H) + (n_occ/n) I on 32 x 32 upper tiles, mirrored.
__global__ void p0_kernel(const double* __restrict__ H, int64_t n, int64_t ldh, int64_t n_occ,
                          const PurifyState* st, double* __restrict__ P, int64_t ldp, int T) {
  __shared__ double tile[32][33];
  int bi, bj;
  upper_tile(blockIdx.x, T, bi, bj);
  const double dn = static_cast<double>(n);
  const double a = st->lam / dn, mu = st->mu, occ = static_cast<double>(n_occ) / dn;
  // SP2 / TRS4: X_0 = (h_max I - H) / (h_max - h_min)
  const bool var = st->method != DMP_METHOD_PM;
  const bool r32 = st->store32 != 0;
  const double hmax = st->h_max, width = st->h_max - st->h_min;
  const int64_t r0 = static_cast<int64_t>(bi) * 32, c0 = static_cast<int64_t>(bj) * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    if (r < n && c < n) tile[y][threadIdx.x] = H[r * ldh + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int x = threadIdx.x;
    const int64_t r = r0 + y, c = c0 + x;
    if (r < n && c < n) {
      double v;
      if (bi == bj) {
        // on the diagonal tile the lower half takes the mirror of the upper half
        const double h = (y <= x) ? tile[y][x] : tile[x][y];
        if (var) {
          v = (r == c) ? (hmax - h) / width : -h / width;
        } else {
          v = (r == c) ? a * (mu - h) + occ : -a * h;
        }
      } else {
        v = var ? -tile[y][x] / width : -a * tile[y][x];
      }
      P[r * ldp + c] = stored_value(v, r32);
    }
  }
  if (bi != bj) {
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
      // write the transposed tile: P[c0 + y][r0 + x] = -a H[r0 + x][c0 + y]
      const int64_t r = c0 + y, c = r0 + threadIdx.x;
      if (r < n && c < n)
        P[r * ldp + c] = stored_value(var ? -tile[threadIdx.x][y] / width : -a * tile[threadIdx.x][y], r32);
    }
  }
}

// Per-block partial measures of the iterate over the upper triangle: rows
// i = blockIdx.x + k * gridDim.x.
//   0: sum P_ii      1: sum X2_ii
//   2: diag P X2     3: upper P X2
//   4: diag (X2-P)^2 5: upper (X2-P)^2
//   6: diag P H      7: upper P H
//   8: diag X2^2      9: upper X2^2      (NQ = 10: SP2 / TRS4)
template <int NQ>
__global__ void __launch_bounds__(256)
measure_kernel(const double* __restrict__ P, int64_t ldp, const double* __restrict__ X2, int64_t ldx,
               const double* __restrict__ H, int64_t ldh, int64_t n, double* __restrict__ part,
               const PurifyState* st) {
  if (st->done) return;
  double d_xx = 0.0, a_xx[4] = {0.0, 0.0, 0.0, 0.0};
  // four independent accumulator sets (entries j, j + 256, j + 512, j + 768 of
  // a step) keep twelve loads in flight per thread; combined in order below
  double a_px[4] = {0.0, 0.0, 0.0, 0.0}, a_id[4] = {0.0, 0.0, 0.0, 0.0}, a_ph[4] = {0.0, 0.0, 0.0, 0.0};
  double d_p = 0.0, d_x = 0.0, d_px = 0.0, d_id = 0.0, d_ph = 0.0;
  const int64_t B = blockDim.x;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double* pr = P + i * ldp;
    const double* xr = X2 + i * ldx;
    const double* hr = H + i * ldh;
    if (threadIdx.x == 0) {
      const double p = pr[i], x = xr[i], h = hr[i];
      d_p += p;
      d_x += x;
      d_px += p * x;
      d_id += (x - p) * (x - p);
      d_ph += p * h;
      if (NQ == 10) d_xx += x * x;
    }
    int64_t j = i + 1 + threadIdx.x;
    for (; j + 3 * B < n; j += 4 * B) {
      double p[4], x[4], h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        p[u] = pr[j + u * B];
        x[u] = xr[j + u * B];
        h[u] = hr[j + u * B];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a_px[u] += p[u] * x[u];
        a_id[u] += (x[u] - p[u]) * (x[u] - p[u]);
        a_ph[u] += p[u] * h[u];
        if (NQ == 10) a_xx[u] += x[u] * x[u];
      }
    }
    for (; j < n; j += B) {
      const double p = pr[j], x = xr[j], h = hr[j];
      a_px[0] += p * x;
      a_id[0] += (x - p) * (x - p);
      a_ph[0] += p * h;
      if (NQ == 10) a_xx[0] += x * x;
    }
  }
  const double u_px = (a_px[0] + a_px[1]) + (a_px[2] + a_px[3]);
  const double u_id = (a_id[0] + a_id[1]) + (a_id[2] + a_id[3]);
  const double u_ph = (a_ph[0] + a_ph[1]) + (a_ph[2] + a_ph[3]);
  const double u_xx = (a_xx[0] + a_xx[1]) + (a_xx[2] + a_xx[3]);
  __shared__ double red[8][NQ];
  double v[NQ];
  v[0] = d_p, v[1] = d_x, v[2] = d_px, v[3] = u_px, v[4] = d_id, v[5] = u_id, v[6] = d_ph, v[7] = u_ph;
  if (NQ == 10) v[NQ - 2] = d_xx, v[NQ - 1] = u_xx;
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < NQ) {
    double t = 0.0;
    for (int ww = 0; ww < 8; ++ww) t += red[ww][threadIdx.x];
    part[static_cast<int64_t>(blockIdx.x) * NQ + threadIdx.x] = t;
  }
}

// Sum the partials in a fixed order and apply the stopping rules; one CTA of
// 256 threads: thread t sums blocks t, t + 256, ... of all NQ measures, then
// warp trees and the eight warps in order. NQ = 8: canonical purification
// (pm_decide); NQ = 10: SP2 / TRS4 (variant_decide).
template <int NQ>
__global__ void __launch_bounds__(256)
measure_final_kernel(const double* __restrict__ part, int nblocks, PurifyState* st) {
  if (st->done) return;
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += part[static_cast<int64_t>(b) * NQ + q];
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  __shared__ double red[8][NQ];
  __shared__ double tot[NQ];
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[threadIdx.x >> 5][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (NQ == 8) {
      pm_decide(st, tot);
    } else {
      variant_decide(st, tot);
    }
  }
}

// Out = alpha X + b2 X2 (SP2 steps), over the full n x n (grid-stride, rows of 256 threads)
__global__ void __launch_bounds__(256)
axpby_kernel(const double* __restrict__ X, int64_t ldx, const double* __restrict__ X2, int64_t ldx2,
             double* __restrict__ out, int64_t ldo, int64_t n, const PurifyState* st) {
  const double a = st->alpha, b = st->b2;
  const bool r32 = st->store32 != 0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
      out[i * ldo + j] = stored_value(a * X[i * ldx + j] + b * X2[i * ldx2 + j], r32);
  }
}

// Z = zd I + zx X + zx2 X2 (the TRS4 factor with F + gamma G = X2 Z)
__global__ void __launch_bounds__(256)
trs4_z_kernel(const double* __restrict__ X, int64_t ldx, const double* __restrict__ X2, int64_t ldx2,
              double* __restrict__ out, int64_t ldo, int64_t n, const PurifyState* st) {
  const double zd = st->zd, zx = st->zx, zx2 = st->zx2;
  const bool r32 = st->store32 != 0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double v = zx * X[i * ldx + j] + zx2 * X2[i * ldx2 + j];
      out[i * ldo + j] = stored_value(j == i ? v + zd : v, r32);
    }
  }
}

// The update weights of a McWeeny step (c = 1/2): alpha = 0, b2 = 3, b3 = -2.
__global__ void refine_weights_kernel(PurifyState* st) {
  st->alpha = 0.0;
  st->b2 = 3.0;
  st->b3 = -2.0;
}

// Per-block partial sums of tr(P H) over the upper triangle: [0] diagonal, [1] strictly upper.
__global__ void __launch_bounds__(256)
energy_kernel(const double* __restrict__ P, int64_t ldp, const double* __restrict__ H, int64_t ldh, int64_t n,
              double* __restrict__ part) {
  double d = 0.0, u = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double* pr = P + i * ldp;
    const double* hr = H + i * ldh;
    if (threadIdx.x == 0) d += pr[i] * hr[i];
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) u += pr[j] * hr[j];
  }
  d = warp_sum(d);
  u = warp_sum(u);
  __shared__ double red[8][2];
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = d;
    red[threadIdx.x >> 5][1] = u;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[static_cast<int64_t>(blockIdx.x) * 2 + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256)
energy_final_kernel(const double* __restrict__ part, int nblocks, PurifyState* st) {
  double d = 0.0, u = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    d += part[2 * b];
    u += part[2 * b + 1];
  }
  d = warp_sum(d);
  u = warp_sum(u);
  __shared__ double red[8][2];
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = d;
    red[threadIdx.x >> 5][1] = u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double td = 0.0, tu = 0.0;
    for (int w = 0; w < 8; ++w) {
      td += red[w][0];
      tu += red[w][1];
    }
    st->energy_refined = td + 2.0 * tu;
  }
}

}  // namespace

cudaError_t launch_measure_variant(const double* X, int64_t ldx, const double* X2, int64_t ldx2, const double* H,
                                   int64_t ldh, int64_t n, double* partials, PurifyState* state, cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  measure_kernel<10><<<kMeasureBlocks, 256, 0, st>>>(X, ldx, X2, ldx2, H, ldh, n, partials, state);
  measure_final_kernel<10><<<1, 256, 0, st>>>(partials, kMeasureBlocks, state);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_axpby(const double* X, int64_t ldx, const double* X2, int64_t ldx2, double* out, int64_t ldo,
                         int64_t n, const PurifyState* state, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  axpby_kernel<<<static_cast<unsigned>(std::min<int64_t>(n, 4 * 152)), 256, 0, st>>>(X, ldx, X2, ldx2, out, ldo, n,
                                                                                     state);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_trs4_z(const double* X, int64_t ldx, const double* X2, int64_t ldx2, double* out, int64_t ldo,
                          int64_t n, const PurifyState* state, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  trs4_z_kernel<<<static_cast<unsigned>(std::min<int64_t>(n, 4 * 152)), 256, 0, st>>>(X, ldx, X2, ldx2, out, ldo,
                                                                                      n, state);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_weights(PurifyState* state, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  refine_weights_kernel<<<1, 1, 0, st>>>(state);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_energy(const double* P, int64_t ldp, const double* H, int64_t ldh, int64_t n, double* partials,
                          PurifyState* state, cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  energy_kernel<<<kMeasureBlocks, 256, 0, st>>>(P, ldp, H, ldh, n, partials);
  energy_final_kernel<<<1, 256, 0, st>>>(partials, kMeasureBlocks, state);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_gershgorin_init(const double* H, int64_t n, int64_t ldh, int64_t n_occ,
                                   double* rowbuf, PurifyState* state, double* P, int64_t ldp,
                                   cudaStream_t st) {
  double* U = rowbuf;
  double* D = rowbuf + n;
  double* Cp = rowbuf + 2 * n;
  int* flag = reinterpret_cast<int*>(rowbuf + 2 * n + static_cast<int64_t>(kColChunks) * n);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  ProfScope prof(DMP_PROF_INIT, st);
  gersh_rows_kernel<<<static_cast<unsigned>(n), kRowThreads, 0, st>>>(H, n, ldh, U, D, flag);
  dim3 cg(static_cast<unsigned>((n + 127) / 128), kColChunks);
  gersh_cols_kernel<<<cg, 128, 0, st>>>(H, n, ldh, Cp);
  gersh_final_kernel<<<1, 1024, 0, st>>>(n, n_occ, U, D, Cp, state, flag);
  const int T = static_cast<int>((n + 31) / 32);
  p0_kernel<<<T * (T + 1) / 2, dim3(32, 8), 0, st>>>(H, n, ldh, n_occ, state, P, ldp, T);
  count_launch(4);
  return cudaGetLastError();
}

size_t gershgorin_rowbuf_bytes(int64_t n) {
  return static_cast<size_t>((2 + kColChunks) * n + 1) * sizeof(double);
}

cudaError_t launch_measure(const double* P, int64_t ldp, const double* X2, int64_t ldx,
                           const double* H, int64_t ldh, int64_t n, double* partials,
                           PurifyState* state, cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  measure_kernel<8><<<kMeasureBlocks, 256, 0, st>>>(P, ldp, X2, ldx, H, ldh, n, partials, state);
  measure_final_kernel<8><<<1, 256, 0, st>>>(partials, kMeasureBlocks, state);
  count_launch(2);
  return cudaGetLastError();
}

}  // namespace dmp
