// Reverse mode through canonical purification: the elementwise and reduction
// kernels of dm_purify_backward. The products (G P, Y P, Z P) run on the same
// executors as the forward.
//
// Step k (c frozen at its forward value, branch frozen; the dependence of c on
// P kept), all matrices symmetric except Y:
//   Y = G P,  Z = Y^T = P G,  YP = G P^2,  ZP = P G P,  X2 = P^2
//   g = alpha G + b2 (Y + Z) + b3 (YP + ZP + YP^T) + (dL/dc) dc/dP
//   dL/dc = alpha' <G, P> + b2' <G, X2> + b3' <Z, X2>     (<G, P^3> = <P G, P^2>)
//   dc/dP = ((2 P - 3 X2) t_d - t_n (I - 2 P)) / t_d^2,  t_d = tr(P - X2), t_n = c t_d
// and the new G is the symmetric part of g (the loss sees P only through
// symmetric matrices, so the symmetric part carries every directional
// derivative along symmetric perturbations).
//
// Initial guess P_0 = (lambda/n)(mu I - H) + (n_occ/n) I, with mu = tr(H)/n
// and lambda = min(n_occ/(h_max - mu), (n - n_occ)/(mu - h_min)) from the
// Gershgorin bounds, whose extreme rows a (max) and b (min) enter through
// h = H_aa + sum_j |H_aj| (and the same with a minus sign for b).

#include "dmp_internal.cuh"

namespace dmp {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Partial sums over all elements, rows i = blockIdx.x + k gridDim.x:
//   0: tr P   1: tr X2   2: <G, P>   3: <G, X2>   4: <Z, X2>
__global__ void __launch_bounds__(256)
adj_reduce_kernel(const double* __restrict__ P, const double* __restrict__ X2, const double* __restrict__ G,
                  const double* __restrict__ Z, int64_t n, double* __restrict__ part) {
  double v[5] = {0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int64_t o = i * n;
    if (threadIdx.x == 0) {
      v[0] += P[o + i];
      v[1] += X2[o + i];
    }
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double p = P[o + j], x = X2[o + j];
      v[2] += G[o + j] * p;
      v[3] += G[o + j] * x;
      v[4] += Z[o + j] * x;
    }
  }
  __shared__ double red[8][5];
#pragma unroll
  for (int q = 0; q < 5; ++q) v[q] = warp_sum(v[q]);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) red[threadIdx.x >> 5][q] = v[q];
  __syncthreads();
  if (threadIdx.x < 5) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[static_cast<int64_t>(blockIdx.x) * 5 + threadIdx.x] = t;
  }
}

// One thread: weights of the frozen step, their c-derivatives and dL/dc.
__global__ void adj_scalars_kernel(const double* __restrict__ part, int nblocks, double c,
                                   AdjScalars* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s[5] = {0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int q = 0; q < 5; ++q) s[q] += part[static_cast<int64_t>(b) * 5 + q];
  double a, b2, b3, da, db2, db3;
  if (c >= 0.5) {
    a = 0.0;
    b2 = (1.0 + c) / c;
    b3 = -1.0 / c;
    da = 0.0;
    db2 = -1.0 / (c * c);
    db3 = 1.0 / (c * c);
  } else {
    const double d = 1.0 - c;
    a = (1.0 - 2.0 * c) / d;
    b2 = (1.0 + c) / d;
    b3 = -1.0 / d;
    da = -1.0 / (d * d);
    db2 = 2.0 / (d * d);
    db3 = -1.0 / (d * d);
  }
  const double td = s[0] - s[1];
  out->alpha = a;
  out->b2 = b2;
  out->b3 = b3;
  out->td = td;
  out->tn = c * td;
  out->dLdc = da * s[2] + db2 * s[3] + db3 * s[4];
}

// G_new = sym(g), one thread per element pair on the upper triangle.
__global__ void adj_step_kernel(const double* __restrict__ G, const double* __restrict__ Y,
                                const double* __restrict__ YP, const double* __restrict__ ZP,
                                const double* __restrict__ P, const double* __restrict__ X2, int64_t n,
                                const AdjScalars* __restrict__ sc, double* __restrict__ Gn) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j < i || j >= n) return;
  const double a = sc->alpha, b2 = sc->b2, b3 = sc->b3;
  const double td = sc->td, tn = sc->tn, k = sc->dLdc / (td * td);
  const int64_t ij = i * n + j, ji = j * n + i;
  const double dij = (i == j) ? 1.0 : 0.0;
  // G, P, X2 are symmetric; Y, YP, ZP are not
  const double dc = ((2.0 * P[ij] - 3.0 * X2[ij]) * td - tn * (dij - 2.0 * P[ij])) * k;
  const double yy = Y[ij] + Y[ji];
  const double gij = a * G[ij] + b2 * yy + b3 * (YP[ij] + ZP[ij] + YP[ji]) + dc;
  const double gji = a * G[ij] + b2 * yy + b3 * (YP[ji] + ZP[ji] + YP[ij]) + dc;
  const double v = 0.5 * (gij + gji);
  Gn[ij] = v;
  Gn[ji] = v;
}

// Symmetric part of a general n x n matrix (leading dimension ld) into dense out.
__global__ void sym_part_kernel(const double* __restrict__ A, int64_t ld, int64_t n, double* __restrict__ out) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j < i || j >= n) return;
  const double v = 0.5 * (A[i * ld + j] + A[j * ld + i]);
  out[i * n + j] = v;
  out[j * n + i] = v;
}

// Partial sums for the initial-guess adjoint: 0: tr G0, 1: <G0, H> (H read as
// its upper triangle mirrored, G0 symmetric).
__global__ void __launch_bounds__(256)
p0_reduce_kernel(const double* __restrict__ G0, const double* __restrict__ H, int64_t ldh, int64_t n,
                 double* __restrict__ part) {
  double tr = 0.0, dg = 0.0, up = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    if (threadIdx.x == 0) {
      tr += G0[i * n + i];
      dg += G0[i * n + i] * H[i * ldh + i];
    }
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) up += G0[i * n + j] * H[i * ldh + j];
  }
  __shared__ double red[8][3];
  tr = warp_sum(tr);
  dg = warp_sum(dg);
  up = warp_sum(up);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = tr;
    red[threadIdx.x >> 5][1] = dg;
    red[threadIdx.x >> 5][2] = up;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    part[static_cast<int64_t>(blockIdx.x) * 3 + threadIdx.x] = t;
  }
}

__global__ void p0_scalars_kernel(const double* __restrict__ part, int nblocks, P0Adjoint* __restrict__ s) {
  if (threadIdx.x != 0) return;
  double tr = 0.0, dg = 0.0, up = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    tr += part[b * 3 + 0];
    dg += part[b * 3 + 1];
    up += part[b * 3 + 2];
  }
  const double n = s->n, lam = s->lam, mu = s->mu;
  const double G0H = dg + 2.0 * up;
  const double dLdlam = (mu * tr - G0H) / n;
  double dLdmu = (lam / n) * tr;
  double dhmax = 0.0, dhmin = 0.0;
  if (s->lam_branch == 1) {
    const double d = (s->h_max - mu) * (s->h_max - mu);
    dLdmu += dLdlam * s->n_occ / d;
    dhmax = -dLdlam * s->n_occ / d;
  } else {
    const double d = (mu - s->h_min) * (mu - s->h_min);
    dLdmu += -dLdlam * (n - s->n_occ) / d;
    dhmin = dLdlam * (n - s->n_occ) / d;
  }
  s->diag_add = dLdmu / n;
  s->dhmax = s->bounds_grad ? dhmax : 0.0;
  s->dhmin = s->bounds_grad ? dhmin : 0.0;
}

// dL/dH (symmetric part): -(lambda/n) G0 + (dL/dmu / n) I + Gershgorin row terms.
__global__ void p0_adjoint_kernel(const double* __restrict__ G0, const double* __restrict__ H, int64_t ldh,
                                  int64_t n, const P0Adjoint* __restrict__ s, double* __restrict__ out,
                                  int64_t ldo) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j < i || j >= n) return;
  const double a = s->lam / s->n;
  double v = -a * G0[i * n + j];
  const int64_t ra = s->row_max, rb = s->row_min;
  const double h = H[i * ldh + j];  // upper triangle, mirrored for (j, i)
  if (i == j) {
    v += s->diag_add;
    if (i == ra) v += s->dhmax;
    if (i == rb) v += s->dhmin;
  } else {
    // the extreme row's radius holds |H_ij| once: half of it on each mirror
    const double sg = (h > 0.0) ? 1.0 : (h < 0.0 ? -1.0 : 0.0);
    if (i == ra || j == ra) v += 0.5 * s->dhmax * sg;
    if (i == rb || j == rb) v -= 0.5 * s->dhmin * sg;
  }
  out[i * ldo + j] = v;
  out[j * ldo + i] = v;
}

}  // namespace

constexpr int kAdjBlocks = 304;

cudaError_t launch_adj_reduce(const double* P, const double* X2, const double* G, const double* Z, int64_t n,
                              double* part, double c, AdjScalars* sc, cudaStream_t st) {
  ProfScope prof(DMP_PROF_MEASURE, st);
  adj_reduce_kernel<<<kAdjBlocks, 256, 0, st>>>(P, X2, G, Z, n, part);
  adj_scalars_kernel<<<1, 32, 0, st>>>(part, kAdjBlocks, c, sc);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_adj_step(const double* G, const double* Y, const double* YP, const double* ZP,
                            const double* P, const double* X2, int64_t n, const AdjScalars* sc, double* Gn,
                            cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(n));
  adj_step_kernel<<<grid, 256, 0, st>>>(G, Y, YP, ZP, P, X2, n, sc, Gn);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sym_part(const double* A, int64_t ld, int64_t n, double* out, cudaStream_t st) {
  ProfScope prof(DMP_PROF_OTHER, st);
  dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(n));
  sym_part_kernel<<<grid, 256, 0, st>>>(A, ld, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_p0_adjoint(const double* G0, const double* H, int64_t ldh, int64_t n, double* part,
                              P0Adjoint* s, double* out, int64_t ldo, cudaStream_t st) {
  ProfScope prof(DMP_PROF_INIT, st);
  p0_reduce_kernel<<<kAdjBlocks, 256, 0, st>>>(G0, H, ldh, n, part);
  p0_scalars_kernel<<<1, 32, 0, st>>>(part, kAdjBlocks, s);
  dim3 grid(static_cast<unsigned>((n + 255) / 256), static_cast<unsigned>(n));
  p0_adjoint_kernel<<<grid, 256, 0, st>>>(G0, H, ldh, n, s, out, ldo);
  count_launch(3);
  return cudaGetLastError();
}

}  // namespace dmp
