// Interface steps of Sec. 2 (steps 3-6), the FP64 residual stencil and the
// layer-gradient reduction.
//
//  * contract_rows / contract_cols: the first half of every transform that is
//    only needed on a few rows -- v next to the interfaces (step 3) is
//    W_x[e,:] V~ W_y^T, and w on the interfaces (step 5) is W_x[p,:] w~ W_y^T;
//    the contraction with one eigenvector row is done here, the remaining
//    short transform by the row-transform kernels.
//  * iface_residual: step 4, r = M f - A v on the interface planes.  v is zero
//    on the interfaces, so only the couplings to the two neighbouring nodes
//    across the interface enter (residual support, Sec. 2).
//  * write_iface: step 7 on the interfaces, u = w there.
//  * stencil_residual: rho = f - M^{-1} A u with the 7-point operator of
//    Eq. (fd)/(fdmtr), for iterative refinement and residual reports.
//  * grad_layers: G_L = sum_{k in L} hhat^z_k sum conj(lam) hhat^x hhat^y u.
#include <algorithm>

#include "hz_convert.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 c, double2 y, double2 acc) {
  return make_double2(fma(c.x, y.x, fma(-c.y, y.y, acc.x)), fma(c.x, y.y, fma(c.y, y.x, acc.y)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// C = double2: FP64 arithmetic; C = float2: FP32 arithmetic (mixed path) on complex128 or
// complex64 data (TV).
// real_coef (FP64): the coefficients are real (their imaginary parts are zero), 2 FMA per term.
template <typename C, typename TV>
__global__ void contract_rows_kernel(const TV* __restrict__ V, double2* __restrict__ out,
                                     const C* __restrict__ coef, const int2* __restrict__ range,
                                     int nrows, int ncols, int nslots, long long nplanes, int real_coef) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = nplanes * nslots * (long long)ncols;
  if (t >= total) return;
  const int j = (int)(t % ncols);
  const long long ps = t / ncols;
  const int s = (int)(ps % nslots);
  const long long plane = ps / nslots;
  const int2 rg = range[s];
  const TV* __restrict__ v = V + plane * (long long)nrows * ncols + j;
  const C* __restrict__ c = coef + (long long)s * nrows;
  if constexpr (sizeof(C) == sizeof(double2)) {
    double2 acc = make_double2(0.0, 0.0);
    if (real_coef) {
      for (int i = rg.x; i < rg.y; ++i) {
        const double ci = c[i].x;
        const double2 x = v[(long long)i * ncols];
        acc.x = fma(ci, x.x, acc.x);
        acc.y = fma(ci, x.y, acc.y);
      }
    } else {
      for (int i = rg.x; i < rg.y; ++i) acc = cfma(c[i], v[(long long)i * ncols], acc);
    }
    out[t] = acc;
  } else {
    float2 acc = make_float2(0.f, 0.f);
    for (int i = rg.x; i < rg.y; ++i) acc = cfma32(c[i], to_c64t(v[(long long)i * ncols]), acc);
    out[t] = to_c128(acc);
  }
}

// FP64: one thread per output (plane, slot, row i) walking its row (the loads of a warp hit
// 32 rows; every line is reused from L1 by the next iterations).  FP32: one warp per
// output, lanes reading the row's range coalesced, then a shuffle reduction in fixed order.
template <typename C, typename TV>
__global__ void contract_cols_kernel(const TV* __restrict__ V, double2* __restrict__ out,
                                     const C* __restrict__ coef, const int2* __restrict__ range,
                                     int nrows, int ncols, int nslots, long long nplanes, int real_coef) {
  constexpr bool F64 = sizeof(C) == sizeof(double2);
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long t = F64 ? gt : gt >> 5;
  const int lane = F64 ? 0 : (int)(threadIdx.x & 31);
  const long long total = nplanes * nslots * (long long)nrows;
  if (t >= total) return;                                  // warp-uniform in the FP32 variant
  const int i = (int)(t % nrows);
  const long long ps = t / nrows;
  const int s = (int)(ps % nslots);
  const long long plane = ps / nslots;
  const int2 rg = range[s];
  const TV* __restrict__ v = V + (plane * nrows + i) * (long long)ncols;
  const C* __restrict__ c = coef + (long long)s * ncols;
  if constexpr (F64) {
    double2 acc = make_double2(0.0, 0.0);
    if (real_coef) {
      for (int j = rg.x; j < rg.y; ++j) {
        const double cj = c[j].x;
        const double2 x = v[j];
        acc.x = fma(cj, x.x, acc.x);
        acc.y = fma(cj, x.y, acc.y);
      }
    } else {
      for (int j = rg.x; j < rg.y; ++j) acc = cfma(c[j], v[j], acc);
    }
    out[t] = acc;
  } else {
    float2 a32 = make_float2(0.f, 0.f);
    for (int j = rg.x + lane; j < rg.y; j += 32) a32 = cfma32(c[j], to_c64t(v[j]), a32);
    for (int o = 16; o > 0; o >>= 1) {
      a32.x += __shfl_down_sync(0xffffffffu, a32.x, o);
      a32.y += __shfl_down_sync(0xffffffffu, a32.y, o);
    }
    if (lane == 0) out[t] = to_c128(a32);
  }
}

// FP32 contraction within rows (mixed path): one warp per (plane, row) takes every slot of the
// row (a slot range is contiguous in the row: consecutive lanes read consecutive columns), so the
// index arithmetic and the row start are shared by the slots; the per-slot sums are reduced
// across the warp at the end.  out[(plane * nslots + s) * nrows + i].
constexpr int kColSlotsMax = 8;
template <typename TV>
__global__ void __launch_bounds__(256) contract_cols_row_kernel(const TV* __restrict__ V, double2* __restrict__ out,
                                                                const float2* __restrict__ coef,
                                                                const int2* __restrict__ range, int nrows,
                                                                int ncols, int nslots, long long nplanes) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = (int)(threadIdx.x & 31);
  if (w >= nplanes * nrows) return;                         // warp-uniform
  const int i = (int)(w % nrows);
  const long long plane = w / nrows;
  const TV* __restrict__ v = V + (plane * nrows + i) * (long long)ncols;
  float2 acc[kColSlotsMax];
#pragma unroll
  for (int s = 0; s < kColSlotsMax; ++s) {
    acc[s] = make_float2(0.f, 0.f);
    if (s < nslots) {
      const int2 rg = range[s];
      const float2* __restrict__ c = coef + (long long)s * ncols;
      for (int j = rg.x + lane; j < rg.y; j += 32) acc[s] = cfma32(c[j], to_c64t(v[j]), acc[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < kColSlotsMax; ++s) {
    if (s < nslots) {
      float2 a32 = acc[s];
      for (int o = 16; o > 0; o >>= 1) {
        a32.x += __shfl_down_sync(0xffffffffu, a32.x, o);
        a32.y += __shfl_down_sync(0xffffffffu, a32.y, o);
      }
      if (lane == 0) out[(plane * nslots + s) * nrows + i] = to_c128(a32);
    }
  }
}

// Step 5 on the mixed path with several interfaces per axis: every slot contracts the
// whole row or column (the whole-axis eigenvector rows), so one pass over V accumulates all
// nslots sums (2 <= nslots <= 8, a compile-time count) in FP32 instead of reading V once
// per slot.

template <int NS, typename TV>
__global__ void contract_rows_multi_kernel(const TV* __restrict__ V, double2* __restrict__ out,
                                           const float2* __restrict__ coef, int nrows, int ncols,
                                           long long nplanes) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nplanes * (long long)ncols) return;
  const int j = (int)(t % ncols);
  const long long plane = t / ncols;
  const TV* __restrict__ v = V + plane * (long long)nrows * ncols + j;
  float2 acc[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int i = 0; i < nrows; ++i) {
    const float2 x = to_c64t(v[(long long)i * ncols]);
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] = cfma32(coef[(long long)q * nrows + i], x, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) out[(plane * NS + q) * (long long)ncols + j] = to_c128(acc[q]);
}

// One warp per (plane, row i): lanes stride over the row, then a shuffle reduction per slot.
template <int NS, typename TV>
__global__ void contract_cols_multi_kernel(const TV* __restrict__ V, double2* __restrict__ out,
                                           const float2* __restrict__ coef, int nrows, int ncols,
                                           long long nplanes) {
  const long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= nplanes * (long long)nrows) return;             // warp-uniform
  const int i = (int)(t % nrows);
  const long long plane = t / nrows;
  const TV* __restrict__ v = V + (plane * nrows + i) * (long long)ncols;
  float2 acc[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int j = lane; j < ncols; j += 32) {
    const float2 x = to_c64t(v[j]);
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] = cfma32(coef[(long long)q * ncols + j], x, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, o);
      acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, o);
    }
    if (lane == 0) out[(plane * NS + q) * (long long)nrows + i] = to_c128(acc[q]);
  }
}

// rX[r][k][p][j] for all j; rY[r][k][q][i] for all i (0 where i is an x-interface).
__global__ void iface_residual_kernel(const IfaceArgs a, const double2* __restrict__ f,
                                      const double2* __restrict__ vX, const double2* __restrict__ vY,
                                      double2* __restrict__ rX, double2* __restrict__ rY) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nXe = (long long)a.nrhs * a.nz * a.nIx * a.ny;
  const long long nYe = (long long)a.nrhs * a.nz * a.nIy * a.nx;
  if (t < nXe) {
    const int j = (int)(t % a.ny);
    const long long rkp = t / a.ny;
    const int p = (int)(rkp % a.nIx);
    const long long rk = rkp / a.nIx;
    const int k = (int)(rk % a.nz);
    const int r = (int)(rk / a.nz);
    const int node = a.xif[p];
    const double2 mzk = a.mz[k], myj = a.my[j];
    const double2 fv = f[(((long long)r * a.nz + k) * a.ny + j) * a.nx + node];
    double2 res = cmul(cmul(a.mx[node], myj), cmul(mzk, fv));
    if (!a.isy[j]) {
      const double2 vl = vX[(rk * 2 * a.nIx + 2 * p) * a.ny + j];
      const double2 vr = vX[(rk * 2 * a.nIx + 2 * p + 1) * a.ny + j];
      double2 nb = cfma(a.ihx[node + 1], vr, cmul(a.ihx[node], vl));
      double2 w = cmul(myj, mzk);
      if (a.sig) { w.x *= a.sig[k]; w.y *= a.sig[k]; }
      res = cfma(w, nb, res);
    }
    rX[t] = res;
  } else if (t < nXe + nYe) {
    const long long u = t - nXe;
    const int i = (int)(u % a.nx);
    const long long rkq = u / a.nx;
    const int q = (int)(rkq % a.nIy);
    const long long rk = rkq / a.nIy;
    const int k = (int)(rk % a.nz);
    const int r = (int)(rk / a.nz);
    if (a.isx[i]) { rY[u] = make_double2(0.0, 0.0); return; }
    const int node = a.yif[q];
    const double2 mzk = a.mz[k], mxi = a.mx[i];
    const double2 fv = f[(((long long)r * a.nz + k) * a.ny + node) * a.nx + i];
    double2 res = cmul(cmul(mxi, a.my[node]), cmul(mzk, fv));
    const double2 vl = vY[(rk * 2 * a.nIy + 2 * q) * a.nx + i];
    const double2 vr = vY[(rk * 2 * a.nIy + 2 * q + 1) * a.nx + i];
    double2 nb = cfma(a.ihy[node + 1], vr, cmul(a.ihy[node], vl));
    double2 w = cmul(mxi, mzk);
    if (a.sig) { w.x *= a.sig[k]; w.y *= a.sig[k]; }
    rY[u] = cfma(w, nb, res);
  }
}

__global__ void write_iface_kernel(const IfaceArgs a, const double2* __restrict__ wX,
                                   const double2* __restrict__ wY, double2* __restrict__ u,
                                   int conj_out, int accumulate) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nXe = (long long)a.nrhs * a.nz * a.nIx * a.ny;
  const long long nYe = (long long)a.nrhs * a.nz * a.nIy * a.nx;
  double2 v;
  long long dst;
  if (t < nXe) {
    const int j = (int)(t % a.ny);
    const long long rkp = t / a.ny;
    const int p = (int)(rkp % a.nIx);
    const long long rk = rkp / a.nIx;
    v = wX[t];
    dst = (rk * a.ny + j) * a.nx + a.xif[p];
  } else if (t < nXe + nYe) {
    const long long s = t - nXe;
    const int i = (int)(s % a.nx);
    if (a.isx[i]) return;
    const long long rkq = s / a.nx;
    const int q = (int)(rkq % a.nIy);
    const long long rk = rkq / a.nIy;
    v = wY[s];
    dst = (rk * a.ny + a.yif[q]) * a.nx + i;
  } else {
    return;
  }
  if (conj_out) v.y = -v.y;
  if (accumulate) {
    double2 o = u[dst];
    v.x += o.x;
    v.y += o.y;
  }
  u[dst] = v;
}

__global__ void adjoint_prep_kernel(const double2* __restrict__ g, double2* __restrict__ out,
                                    const double2* __restrict__ imx, const double2* __restrict__ imy,
                                    const double2* __restrict__ imz, int nx, int ny, int nz,
                                    long long total) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int i = (int)(t % nx);
  const long long q = t / nx;
  const int j = (int)(q % ny);
  const int k = (int)((q / ny) % nz);
  double2 v = g[t];
  v.y = -v.y;
  out[t] = cmul(cmul(v, imx[i]), cmul(imy[j], imz[k]));
}

// Gradient in the right-hand side: out = conj(mx_i my_j mz_k) lam (out may alias lam).
__global__ void grad_rhs_kernel(const double2* lam, double2* out, const double2* __restrict__ mx,
                                const double2* __restrict__ my, const double2* __restrict__ mz, int nx, int ny,
                                int nz, long long total) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int i = (int)(t % nx);
  const long long q = t / nx;
  const int j = (int)(q % ny);
  const int k = (int)((q / ny) % nz);
  double2 w = cmul(mx[i], cmul(my[j], mz[k]));
  w.y = -w.y;
  out[t] = cmul(w, lam[t]);
}

__global__ void conj_kernel(double2* __restrict__ u, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) u[t].y = -u[t].y;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < NT / 32; ++q) s += sh[q];
  return s;
}

constexpr int ST = 256;
constexpr int SEPT = 4;                    // stencil elements per thread

// r = f - M^{-1} A u with the 7-point operator of Eq. (fd), divided by the weights:
//   M^{-1} A u = sigma_k (Kx u / mx + Ky u / my) + Tz u / mz.
// grid (CTAs per plane, nrhs * nz): one plane (r, k) per blockIdx.y, so the z-row of the
// operator and the weight |mz_k|^2 are CTA constants.  Every term is one FMA into the
// accumulator that starts at f (real off-diagonal coefficients -- rows whose steps are
// real -- take two FP64 operations, complex ones four); the centre coefficient
// sigma_k cxy + tz1 is formed first.  ~21 FP64 operations per unknown for real rows.
template <bool SIGMA>
__global__ void __launch_bounds__(ST) stencil_kernel(const StencilArgs a, const double2* __restrict__ f,
                                                     const double2* __restrict__ u,
                                                     double2* __restrict__ rho,
                                                     double* __restrict__ partial, int fnorm, int rk0) {
  __shared__ double sh[ST / 32];
  const int rk = rk0 + blockIdx.y;
  const int k = rk % a.nz;
  const long long nxy = (long long)a.nx * a.ny;
  const long long base = (long long)rk * nxy;
  const double2* __restrict__ ur = u + base;
  const double2* __restrict__ fr = f + base;
  const double2 tz0 = a.tzs[3 * k], tz1 = a.tzs[3 * k + 1], tz2 = a.tzs[3 * k + 2];
  const bool realz = a.rz[k] != 0;
  const double s = SIGMA ? a.sig[k] : 1.0;
  const bool has_dn = k > 0, has_up = k < a.nz - 1;
  double nr2 = 0.0, nf2 = 0.0;
#pragma unroll
  for (int e = 0; e < SEPT; ++e) {
    const int t = ((int)blockIdx.x * SEPT + e) * ST + (int)threadIdx.x;   // in-plane index (< 2^31)
    if (t >= nxy) break;
    const int j = t / a.nx, i = t - j * a.nx;
    const double2 uc = ur[t];
    const double2 fv = fr[t];
    const double2 cx = a.cxy[t];
    // centre: acc = f - (sigma cxy + tz1) u
    double2 c;
    if (SIGMA) c = make_double2(fma(s, cx.x, tz1.x), fma(s, cx.y, tz1.y));
    else c = make_double2(cx.x + tz1.x, cx.y + tz1.y);
    double2 acc = make_double2(fma(-c.x, uc.x, fma(c.y, uc.y, fv.x)), fma(-c.x, uc.y, fma(-c.y, uc.x, fv.y)));
    // horizontal neighbours (scaled by sigma_k): into hz, which is acc itself when sigma = 1
    double2 hz = SIGMA ? make_double2(0.0, 0.0) : acc;
    const double2* kx = a.kxs + 3 * i;
    const double2* ky = a.kys + 3 * j;
    if (a.rx[i]) {
      if (i > 0) { const double2 v = ur[t - 1]; hz.x = fma(-kx[0].x, v.x, hz.x); hz.y = fma(-kx[0].x, v.y, hz.y); }
      if (i < a.nx - 1) { const double2 v = ur[t + 1]; hz.x = fma(-kx[2].x, v.x, hz.x); hz.y = fma(-kx[2].x, v.y, hz.y); }
    } else {
      if (i > 0) hz = cfma(make_double2(-kx[0].x, -kx[0].y), ur[t - 1], hz);
      if (i < a.nx - 1) hz = cfma(make_double2(-kx[2].x, -kx[2].y), ur[t + 1], hz);
    }
    if (a.ry[j]) {
      if (j > 0) { const double2 v = ur[t - a.nx]; hz.x = fma(-ky[0].x, v.x, hz.x); hz.y = fma(-ky[0].x, v.y, hz.y); }
      if (j < a.ny - 1) { const double2 v = ur[t + a.nx]; hz.x = fma(-ky[2].x, v.x, hz.x); hz.y = fma(-ky[2].x, v.y, hz.y); }
    } else {
      if (j > 0) hz = cfma(make_double2(-ky[0].x, -ky[0].y), ur[t - a.nx], hz);
      if (j < a.ny - 1) hz = cfma(make_double2(-ky[2].x, -ky[2].y), ur[t + a.nx], hz);
    }
    if (SIGMA) {
      acc.x = fma(s, hz.x, acc.x);
      acc.y = fma(s, hz.y, acc.y);
    } else {
      acc = hz;
    }
    if (realz) {
      if (has_dn) { const double2 v = ur[t - nxy]; acc.x = fma(-tz0.x, v.x, acc.x); acc.y = fma(-tz0.x, v.y, acc.y); }
      if (has_up) { const double2 v = ur[t + nxy]; acc.x = fma(-tz2.x, v.x, acc.x); acc.y = fma(-tz2.x, v.y, acc.y); }
    } else {
      if (has_dn) acc = cfma(make_double2(-tz0.x, -tz0.y), ur[t - nxy], acc);
      if (has_up) acc = cfma(make_double2(-tz2.x, -tz2.y), ur[t + nxy], acc);
    }
    if (rho) rho[base + t] = acc;
    const double w2 = a.w2xy[t];
    nr2 = fma(w2, fma(acc.x, acc.x, acc.y * acc.y), nr2);
    if (fnorm) nf2 = fma(w2, fma(fv.x, fv.x, fv.y * fv.y), nf2);
  }
  const double wz = a.w2z[k];
  const double s1 = block_sum<ST>(nr2, sh) * wz;
  const double s2 = fnorm ? block_sum<ST>(nf2, sh) * wz : 0.0;
  if (threadIdx.x == 0) {
    const long long part = (long long)rk * gridDim.x + blockIdx.x;   // = (r * nz + k) * gx + bx
    partial[part * 2 + 0] = s1;
    partial[part * 2 + 1] = s2;
  }
}

// out[2r + c] = sum_p partial[r][p][c]: each thread sums a fixed stride of the parts, then a
// fixed-order tree (deterministic for a given launch shape).
__global__ void __launch_bounds__(ST) finish_norms_kernel(const double* __restrict__ partial, int nparts,
                                                          double* out) {
  __shared__ double sh[2][ST];
  const int r = blockIdx.x;
  double s0 = 0.0, s1 = 0.0;
  for (int p = threadIdx.x; p < nparts; p += ST) {
    s0 += partial[((long long)r * nparts + p) * 2 + 0];
    s1 += partial[((long long)r * nparts + p) * 2 + 1];
  }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = ST / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * r] = sh[0][0];
    out[2 * r + 1] = sh[1][0];
  }
}

// grid (nparts, nz): CTA sums conj(lam) mx my u over a slice of (r, j, i) of plane k.
__global__ void __launch_bounds__(ST) grad_kernel(const double2* __restrict__ u,
                                                  const double2* __restrict__ lam,
                                                  const double2* __restrict__ mx,
                                                  const double2* __restrict__ my, int nx, int ny,
                                                  int nz, int nrhs, double2* __restrict__ partial) {
  __shared__ double sh[ST / 32];
  const int k = blockIdx.y;
  const long long nxy = (long long)nx * ny;
  const long long n = nxy * nrhs;
  double sr = 0.0, si = 0.0;
  for (long long t = blockIdx.x * (long long)ST + threadIdx.x; t < n; t += (long long)gridDim.x * ST) {
    const int r = (int)(t / nxy);
    const long long pos = t - (long long)r * nxy;
    const int j = (int)(pos / nx), i = (int)(pos - (long long)j * nx);
    const long long idx = ((long long)r * nz + k) * nxy + pos;
    double2 l = lam[idx];
    l.y = -l.y;
    const double2 v = cmul(cmul(l, u[idx]), cmul(mx[i], my[j]));
    sr += v.x;
    si += v.y;
  }
  const double a = block_sum<ST>(sr, sh);
  const double b = block_sum<ST>(si, sh);
  if (threadIdx.x == 0) partial[(long long)k * gridDim.x + blockIdx.x] = make_double2(a, b);
}

__global__ void grad_finish_kernel(const double2* __restrict__ partial, int nparts,
                                   const double2* __restrict__ mz, const int* __restrict__ z_begin,
                                   int nlayers, double2* __restrict__ G) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlayers) return;
  double2 g = make_double2(0.0, 0.0);
  for (int k = z_begin[L]; k < z_begin[L + 1]; ++k) {
    double2 pk = make_double2(0.0, 0.0);
    for (int p = 0; p < nparts; ++p) pk = cadd(pk, partial[(long long)k * nparts + p]);
    g = cfma(mz[k], pk, g);
  }
  G[L] = g;
}

unsigned blocks_for(long long n, int T) { return (unsigned)((n + T - 1) / T); }

}  // namespace

template <typename C, typename TV>
void contract_rows_t(const TV* V, double2* out, const C* coef, const int2* range, int nrows, int ncols,
                     int nslots, long long nplanes, cudaStream_t st, int real_coef = 0) {
  const long long n = nplanes * nslots * (long long)ncols;
  if (n == 0) return;
  contract_rows_kernel<C, TV><<<blocks_for(n, 128), 128, 0, st>>>(V, out, coef, range, nrows, ncols, nslots,
                                                                 nplanes, real_coef);
  count_launch();
}

template <typename C, typename TV>
void contract_cols_t(const TV* V, double2* out, const C* coef, const int2* range, int nrows, int ncols,
                     int nslots, long long nplanes, cudaStream_t st, int real_coef = 0) {
  const long long n = nplanes * nslots * (long long)nrows;
  if (n == 0) return;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (nslots <= kColSlotsMax) {                            // FP32: one warp per row, all slots
      contract_cols_row_kernel<TV><<<blocks_for(nplanes * nrows * 32, 256), 256, 0, st>>>(
          V, out, coef, range, nrows, ncols, nslots, nplanes);
      count_launch();
      return;
    }
  }
  const long long threads = sizeof(C) == sizeof(double2) ? n : n * 32;   // FP32: one warp per output
  contract_cols_kernel<C, TV><<<blocks_for(threads, 256), 256, 0, st>>>(V, out, coef, range, nrows, ncols,
                                                                       nslots, nplanes, real_coef);
  count_launch();
}

template <int NS, typename TV>
void contract_all_t(bool rows, const TV* V, double2* out, const float2* coef, int nrows, int ncols,
                    long long nplanes, cudaStream_t st) {
  if (rows) {
    const long long n = nplanes * (long long)ncols;
    if (n == 0) return;
    contract_rows_multi_kernel<NS, TV><<<blocks_for(n, 128), 128, 0, st>>>(V, out, coef, nrows, ncols, nplanes);
  } else {
    const long long n = nplanes * (long long)nrows;
    if (n == 0) return;
    contract_cols_multi_kernel<NS, TV><<<blocks_for(n * 32, 256), 256, 0, st>>>(V, out, coef, nrows, ncols,
                                                                              nplanes);
  }
  count_launch();
}

template <typename TV>
bool contract_all_any(bool rows, const TV* V, double2* out, const float2* coef, int nrows, int ncols,
                      int nslots, long long nplanes, cudaStream_t st) {
  switch (nslots) {        // the slot count is a compile-time constant of the kernels
    case 2: contract_all_t<2>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    case 3: contract_all_t<3>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    case 4: contract_all_t<4>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    case 5: contract_all_t<5>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    case 6: contract_all_t<6>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    case 7: contract_all_t<7>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    case 8: contract_all_t<8>(rows, V, out, coef, nrows, ncols, nplanes, st); return true;
    default: return false;
  }
}

bool contract_all(bool rows, const double2* V, double2* out, const float2* coef, int nrows, int ncols,
                  int nslots, long long nplanes, cudaStream_t st) {
  return contract_all_any(rows, V, out, coef, nrows, ncols, nslots, nplanes, st);
}
bool contract_all(bool rows, const float2* V, double2* out, const float2* coef, int nrows, int ncols,
                  int nslots, long long nplanes, cudaStream_t st) {
  return contract_all_any(rows, V, out, coef, nrows, ncols, nslots, nplanes, st);
}

void contract_rows(const double2* V, double2* out, const double2* coef, const int2* range, int nrows,
                   int ncols, int nslots, long long nplanes, cudaStream_t st, bool real_coef) {
  contract_rows_t(V, out, coef, range, nrows, ncols, nslots, nplanes, st, real_coef ? 1 : 0);
}
void contract_rows(const double2* V, double2* out, const float2* coef, const int2* range, int nrows,
                   int ncols, int nslots, long long nplanes, cudaStream_t st) {
  contract_rows_t(V, out, coef, range, nrows, ncols, nslots, nplanes, st);
}
void contract_rows(const float2* V, double2* out, const float2* coef, const int2* range, int nrows,
                   int ncols, int nslots, long long nplanes, cudaStream_t st) {
  contract_rows_t(V, out, coef, range, nrows, ncols, nslots, nplanes, st);
}
void contract_cols(const double2* V, double2* out, const double2* coef, const int2* range, int nrows,
                   int ncols, int nslots, long long nplanes, cudaStream_t st, bool real_coef) {
  contract_cols_t(V, out, coef, range, nrows, ncols, nslots, nplanes, st, real_coef ? 1 : 0);
}
void contract_cols(const double2* V, double2* out, const float2* coef, const int2* range, int nrows,
                   int ncols, int nslots, long long nplanes, cudaStream_t st) {
  contract_cols_t(V, out, coef, range, nrows, ncols, nslots, nplanes, st);
}
void contract_cols(const float2* V, double2* out, const float2* coef, const int2* range, int nrows,
                   int ncols, int nslots, long long nplanes, cudaStream_t st) {
  contract_cols_t(V, out, coef, range, nrows, ncols, nslots, nplanes, st);
}

void iface_residual(const IfaceArgs& a, const double2* f, const double2* vX, const double2* vY,
                    double2* rX, double2* rY, cudaStream_t st) {
  const long long n = (long long)a.nrhs * a.nz * ((long long)a.nIx * a.ny + (long long)a.nIy * a.nx);
  if (n == 0) return;
  iface_residual_kernel<<<blocks_for(n, 128), 128, 0, st>>>(a, f, vX, vY, rX, rY);
  count_launch();
}

void write_iface(const IfaceArgs& a, const double2* wX, const double2* wY, double2* u, int conj_out,
                 int accumulate, cudaStream_t st) {
  const long long n = (long long)a.nrhs * a.nz * ((long long)a.nIx * a.ny + (long long)a.nIy * a.nx);
  if (n == 0) return;
  write_iface_kernel<<<blocks_for(n, 128), 128, 0, st>>>(a, wX, wY, u, conj_out, accumulate);
  count_launch();
}

void adjoint_prep(const double2* g, double2* out, const double2* imx, const double2* imy,
                  const double2* imz, int nx, int ny, int nz, int nrhs, cudaStream_t st) {
  const long long n = (long long)nx * ny * nz * nrhs;
  if (n == 0) return;
  adjoint_prep_kernel<<<blocks_for(n, 256), 256, 0, st>>>(g, out, imx, imy, imz, nx, ny, nz, n);
  count_launch();
}

void grad_rhs(const double2* lam, double2* out, const double2* mx, const double2* my, const double2* mz,
              int nx, int ny, int nz, int nrhs, cudaStream_t st) {
  const long long n = (long long)nx * ny * nz * nrhs;
  if (n == 0) return;
  grad_rhs_kernel<<<blocks_for(n, 256), 256, 0, st>>>(lam, out, mx, my, mz, nx, ny, nz, n);
  count_launch();
}

void conj_inplace(double2* u, long long n, cudaStream_t st) {
  if (n <= 0) return;
  conj_kernel<<<blocks_for(n, 256), 256, 0, st>>>(u, n);
  count_launch();
}

int stencil_parts(const StencilArgs& a) {
  const long long nxy = (long long)a.nx * a.ny;
  const long long gx = (nxy + (long long)ST * SEPT - 1) / ((long long)ST * SEPT);
  return (int)(gx * a.nz);
}

void stencil_residual(const StencilArgs& a, const double2* f, const double2* u, double2* rho,
                      double* partial, int fnorm, cudaStream_t st) {
  const long long nxy = (long long)a.nx * a.ny;
  const unsigned gx = (unsigned)((nxy + (long long)ST * SEPT - 1) / ((long long)ST * SEPT));
  const int planes = a.nrhs * a.nz;
  for (int rk0 = 0; rk0 < planes; rk0 += 65535) {
    dim3 grid(gx, std::min(65535, planes - rk0));
    if (a.sig) stencil_kernel<true><<<grid, ST, 0, st>>>(a, f, u, rho, partial, fnorm, rk0);
    else stencil_kernel<false><<<grid, ST, 0, st>>>(a, f, u, rho, partial, fnorm, rk0);
    count_launch();
  }
}

void finish_norms(const double* partial, int nparts, int nrhs, double* out, cudaStream_t st) {
  finish_norms_kernel<<<nrhs, ST, 0, st>>>(partial, nparts, out);
  count_launch();
}

int grad_parts(int nx, int ny, int nrhs) {
  const long long n = (long long)nx * ny * nrhs;
  long long parts = (n + ST * 8 - 1) / (ST * 8);
  if (parts > 64) parts = 64;
  return parts < 1 ? 1 : (int)parts;
}

void grad_layers(const double2* u, const double2* lam, const double2* mx, const double2* my,
                 const double2* mz, const int* z_begin, int nlayers, int nx, int ny, int nz, int nrhs,
                 double2* partial, int nparts, double2* G, cudaStream_t st) {
  dim3 grid(nparts, nz);
  grad_kernel<<<grid, ST, 0, st>>>(u, lam, mx, my, nx, ny, nz, nrhs, partial);
  count_launch();
  grad_finish_kernel<<<(nlayers + 63) / 64, 64, 0, st>>>(partial, nparts, mz, z_begin, nlayers, G);
  count_launch();
}

}  // namespace hz
