// Mode-wise tridiagonal solves along z (steps 2, 5 and 6 of Sec. 2).
//
// After the x/y eigen-transforms every mode (l, m) of a block decouples into
// one complex-symmetric tridiagonal system of length Nz (Eq. (fdmtrprjfr)):
//     (Tz + s_lm S_z) x = M_z f~,   s_lm = lambda_l + mu_m,   S_z = diag(sigma_k hhat^z_k),
// and the global interface system Eq. (fdmtrprjfrerr) has the same form with the
// whole-axis eigenvalues.  One thread owns one mode and sweeps z (Thomas
// elimination without pivoting); adjacent threads own adjacent modes, so every
// z step is a coalesced access of the [k][i][j] mode layout.
//
// The elimination factors depend only on the mode and the frequency, so they
// are computed once per plan/frequency (zfactor) and the per-solve sweep is
//   forward  y_k = (rhs_k - cm_k y_{k-1}) P_k,   back  x_k = y_k - Q_k x_{k+1},
// with P_k = fold_k / d_k, Q_k = c_{k+1} / d_k, cm_k = c_k / fold_k, d_k the
// pivots.  The forward results are kept in the output array and overwritten by
// the back sweep.  FP64 throughout.
#include "hz_internal.h"

namespace hz {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// b - c * y
__device__ __forceinline__ double2 csub_mul(double2 b, double2 c, double2 y) {
  return make_double2(fma(-c.x, y.x, fma(c.y, y.y, b.x)), fma(-c.x, y.y, fma(-c.y, y.x, b.y)));
}
// acc + c * y
__device__ __forceinline__ double2 cfma(double2 c, double2 y, double2 acc) {
  return make_double2(fma(c.x, y.x, fma(-c.y, y.y, acc.x)), fma(c.x, y.y, fma(c.y, y.x, acc.y)));
}

template <int MODE, bool REALCM>
__global__ void __launch_bounds__(128) zsolve_kernel(const ZSolveArgs a) {
  const long long plane = (long long)a.nx * a.ny;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= plane * a.nrhs) return;
  const int r = (int)(tid / plane);
  const long long pos = tid - (long long)r * plane;
  const int i = (int)(pos / a.ny), j = (int)(pos - (long long)i * a.ny);
  if (MODE != Z_GLOBAL && (a.skip_i[i] | a.skip_j[j])) return;
  const long long rs = plane * a.nz;
  const double2* __restrict__ rhs = a.rhs + r * rs + pos;
  double2* __restrict__ out = a.out + r * rs + pos;
  const double2* __restrict__ P = a.P + pos;
  const double2* __restrict__ Q = a.Q + pos;
  const double2* __restrict__ cm = a.cm;

  // pass B: boundary coefficients of this mode (sigma_k applied per k)
  int pl = -1, pr = -1, ql = -1, qr = -1;
  double2 cxl = {0, 0}, cxr = {0, 0}, cyl = {0, 0}, cyr = {0, 0};
  if (MODE == Z_PASS_B) {
    pl = a.gxl[i]; pr = a.gxr[i]; ql = a.gyl[j]; qr = a.gyr[j];
    if (pl >= 0) cxl = a.cxl[i];
    if (pr >= 0) cxr = a.cxr[i];
    if (ql >= 0) cyl = a.cyl[j];
    if (qr >= 0) cyr = a.cyr[j];
  }

  double2 y = make_double2(0.0, 0.0);
#pragma unroll 4
  for (int k = 0; k < a.nz; ++k) {
    double2 b;
    if (MODE == Z_GLOBAL) {
      b = make_double2(0.0, 0.0);
      const long long base = ((long long)r * a.nz + k);
      for (int p = 0; p < a.nIx; ++p)
        b = cfma(a.WgxI[(long long)p * a.nx + i], a.aX[(base * a.nIx + p) * a.ny + j], b);
      for (int q = 0; q < a.nIy; ++q)
        b = cfma(a.WgyI[(long long)q * a.ny + j], a.bY[(base * a.nIy + q) * a.nx + i], b);
    } else {
      b = rhs[k * plane];
      if (MODE == Z_PASS_B) {
        const long long base = ((long long)r * a.nz + k);
        double2 g = make_double2(0.0, 0.0);
        if (pl >= 0) g = cfma(cxl, a.alphaX[(base * a.nIx + pl) * a.ny + j], g);
        if (pr >= 0) g = cfma(cxr, a.alphaX[(base * a.nIx + pr) * a.ny + j], g);
        if (ql >= 0) g = cfma(cyl, a.alphaY[(base * a.nIy + ql) * a.nx + i], g);
        if (qr >= 0) g = cfma(cyr, a.alphaY[(base * a.nIy + qr) * a.nx + i], g);
        if (a.sig) {
          const double s = a.sig[k];
          b.x = fma(s, g.x, b.x);
          b.y = fma(s, g.y, b.y);
        } else {
          b.x += g.x;
          b.y += g.y;
        }
      }
    }
    const double2 c = cm[k];
    double2 t;
    if (REALCM)
      t = make_double2(fma(-c.x, y.x, b.x), fma(-c.x, y.y, b.y));
    else
      t = csub_mul(b, c, y);
    y = cmul(t, P[k * plane]);
    out[k * plane] = y;
  }
  double2 x = y;
#pragma unroll 4
  for (int k = a.nz - 2; k >= 0; --k) {
    const double2 yk = out[k * plane];
    x = csub_mul(yk, Q[k * plane], x);
    out[k * plane] = x;
  }
}

__global__ void zfactor_kernel(double2* __restrict__ P, double2* __restrict__ Q,
                               const double2* __restrict__ lamx, const double2* __restrict__ lamy,
                               const signed char* __restrict__ skip_i,
                               const signed char* __restrict__ skip_j, const double2* __restrict__ tzd,
                               const double2* __restrict__ szs, const double2* __restrict__ coff,
                               const double2* __restrict__ fold, int nx, int ny, int nz,
                               unsigned long long* min_pivot_bits, int* status) {
  const long long plane = (long long)nx * ny;
  const long long pos = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (pos >= plane) return;
  const int i = (int)(pos / ny), j = (int)(pos - (long long)i * ny);
  if (skip_i && (skip_i[i] | skip_j[j])) return;
  const double2 s = make_double2(lamx[i].x + lamy[j].x, lamx[i].y + lamy[j].y);
  double2 e_prev = make_double2(0.0, 0.0);
  double minpiv = 1.0 / 0.0;
  bool bad = false;
  for (int k = 0; k < nz; ++k) {
    double2 d = tzd[k];
    const double2 sk = cmul(s, szs[k]);
    d.x += sk.x;
    d.y += sk.y;
    if (k > 0) {
      const double2 c = coff[k];
      d = csub_mul(d, cmul(c, c), e_prev);
      Q[(long long)(k - 1) * plane + pos] = cmul(c, e_prev);
    }
    const double den = d.x * d.x + d.y * d.y;
    const double mag = sqrt(den);
    if (!(mag > 0.0) || !isfinite(mag)) bad = true;
    minpiv = fmin(minpiv, mag);
    const double inv = 1.0 / den;
    const double2 e = make_double2(d.x * inv, -d.y * inv);
    P[(long long)k * plane + pos] = fold ? cmul(fold[k], e) : e;
    e_prev = e;
  }
  Q[(long long)(nz - 1) * plane + pos] = make_double2(0.0, 0.0);
  if (bad) atomicExch(status, (int)HZ_ERR_SINGULAR);
  if (isfinite(minpiv)) atomicMin(min_pivot_bits, (unsigned long long)__double_as_longlong(minpiv));
}

}  // namespace

void zsolve(int mode, const ZSolveArgs& a, cudaStream_t st) {
  const long long n = (long long)a.nx * a.ny * a.nrhs;
  if (n == 0) return;
  const int T = 128;
  const unsigned grid = (unsigned)((n + T - 1) / T);
  if (mode == Z_PASS_A) {
    if (a.real_cm) zsolve_kernel<Z_PASS_A, true><<<grid, T, 0, st>>>(a);
    else zsolve_kernel<Z_PASS_A, false><<<grid, T, 0, st>>>(a);
  } else if (mode == Z_PASS_B) {
    if (a.real_cm) zsolve_kernel<Z_PASS_B, true><<<grid, T, 0, st>>>(a);
    else zsolve_kernel<Z_PASS_B, false><<<grid, T, 0, st>>>(a);
  } else {
    if (a.real_cm) zsolve_kernel<Z_GLOBAL, true><<<grid, T, 0, st>>>(a);
    else zsolve_kernel<Z_GLOBAL, false><<<grid, T, 0, st>>>(a);
  }
  count_launch();
}

void zfactor(double2* P, double2* Q, const double2* lamx, const double2* lamy,
             const signed char* skip_i, const signed char* skip_j, const double2* tzd,
             const double2* szs, const double2* coff, const double2* fold, int nx, int ny, int nz,
             unsigned long long* min_pivot_bits, int* status, cudaStream_t st) {
  const long long n = (long long)nx * ny;
  const int T = 128;
  zfactor_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(P, Q, lamx, lamy, skip_i, skip_j, tzd, szs,
                                                           coff, fold, nx, ny, nz, min_pivot_bits,
                                                           status);
  count_launch();
}

}  // namespace hz
