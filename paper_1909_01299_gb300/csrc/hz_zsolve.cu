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
// The right-hand sides of the global pass (r~ of step 5) and the boundary term of
// pass B (g~ of step 6) are rank-|I| outer products of interface data.  On the FP64 path
// they are formed by fully parallel kernels (global_rhs, boundary_rhs); on the mixed path
// (FP32 sums of complex64 interface data) the sweep forms them itself, term by term in the
// same order, so that no complex64 volume is written and read back.  The elimination factors
// depend only on the mode and the frequency, so they are computed once per plan/frequency
// (zfactor) and the per-solve sweep is
//   forward  y_k = (rhs_k - cm_k y_{k-1}) P_k,   back  x_k = y_k - Q_k x_{k+1},
// with P_k = fold_k / d_k, Q_k = c_{k+1} / d_k, cm_k = c_k / fold_k, d_k the
// pivots.  The forward results are kept in the output array and overwritten by
// the back sweep.  The elimination is FP64 throughout; on the mixed path the
// right-hand side and the result are stored as complex64 (they carry the FP32
// accuracy of the tensor-core transforms that produce and consume them) and the
// forward values go to an FP64 scratch array instead.
#include <algorithm>
#include <type_traits>

#include "hz_convert.cuh"
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
// acc + c * y with a real c
__device__ __forceinline__ double2 rfma(double c, double2 y, double2 acc) {
  return make_double2(fma(c, y.x, acc.x), fma(c, y.y, acc.y));
}

// Per-thread constants of a generated right-hand side: kind 1, the thread's coefficients
// wx32[p][i] and wy32[q][j]; kind 2, the interface indices and coefficients of its block edges.
struct GenThread {
  float2 wx[kGenMaxIface], wy[kGenMaxIface];
  int pl = -1, pr = -1, ql = -1, qr = -1;
  float2 cl, cr, dl, dr;
};

// GEN: 0 read rhs32; 2 rhs32 plus the boundary term (kind 2); 10 + NI the global right-hand
// side (kind 1) with NI = max(nIx, nIy) <= kGenMaxIface terms per axis, unrolled at compile
// time (terms past nIx or nIy are skipped by a uniform test).
template <int GEN> __host__ __device__ constexpr int gen_terms() { return GEN > 10 ? GEN - 10 : 0; }

template <int GEN>
__device__ __forceinline__ GenThread gen_thread(const ZSolveArgs& a, int i, int j) {
  GenThread t;
  const ZRhsGen& g = a.gen;
  constexpr int NI = gen_terms<GEN>();
  if constexpr (NI > 0) {
#pragma unroll
    for (int p = 0; p < NI; ++p) {
      t.wx[p] = p < g.nIx ? g.wx32[(long long)p * a.nx + i] : make_float2(0.f, 0.f);
      t.wy[p] = p < g.nIy ? g.wy32[(long long)p * a.ny + j] : make_float2(0.f, 0.f);
    }
  } else if constexpr (GEN == 2) {
    t.pl = g.gxl[i]; t.pr = g.gxr[i]; t.ql = g.gyl[j]; t.qr = g.gyr[j];
    t.cl = g.cxl32[i]; t.cr = g.cxr32[i]; t.dl = g.cyl32[j]; t.dr = g.cyr32[j];
  }
  return t;
}

// Complex64 right-hand side of plane k of RHS r at mode (i, j), element idx of rhs32, as FP64:
// the FP32 sums of global_rhs_kernel and boundary_rhs_kernel, term by term in the same order.
template <int GEN>
__device__ __forceinline__ double2 c64_rhs(const ZSolveArgs& a, const GenThread& gt, long long idx, int r, int k,
                                           int i, int j) {
  constexpr int NI = gen_terms<GEN>();
  if constexpr (GEN == 0) {
    return to_c128(a.rhs32[idx]);
  } else {
    const ZRhsGen& g = a.gen;
    const long long rk = (long long)r * a.nz + k;
    float2 s = make_float2(0.f, 0.f);
    if constexpr (NI > 0) {
      const float2* ax = g.aX32 + rk * g.nIx * a.ny + j;
      const float2* by = g.bY32 + rk * g.nIy * a.nx + i;
      float2 vx[NI], vy[NI];
#pragma unroll
      for (int p = 0; p < NI; ++p) {
        if (p < g.nIx) vx[p] = ax[(long long)p * a.ny];
        if (p < g.nIy) vy[p] = by[(long long)p * a.nx];
      }
#pragma unroll
      for (int p = 0; p < NI; ++p)
        if (p < g.nIx) s = cfma32(gt.wx[p], vx[p], s);
#pragma unroll
      for (int p = 0; p < NI; ++p)
        if (p < g.nIy) s = cfma32(gt.wy[p], vy[p], s);
      return to_c128(s);
    } else {
      const float2* ax = g.aX32 + rk * g.nIx * a.ny + j;
      const float2* ay = g.bY32 + rk * g.nIy * a.nx + i;
      if (gt.pl >= 0) s = cfma32(gt.cl, ax[(long long)gt.pl * a.ny], s);
      if (gt.pr >= 0) s = cfma32(gt.cr, ax[(long long)gt.pr * a.ny], s);
      if (gt.ql >= 0) s = cfma32(gt.dl, ay[(long long)gt.ql * a.nx], s);
      if (gt.qr >= 0) s = cfma32(gt.dr, ay[(long long)gt.qr * a.nx], s);
      const float2 f32 = a.rhs32[idx];
      const double sg = g.sig ? g.sig[k] : 1.0;
      const float s32 = sg == 1.0 ? 1.f : f64_to_f32_trunc(sg);
      return to_c128(make_float2(fmaf(s32, s.x, f32.x), fmaf(s32, s.y, f32.y)));
    }
  }
}

// RB right-hand sides per thread share each factor load and give the sweep RB independent
// dependency chains.  C64: complex64 right-hand side and result (mixed path); the forward
// values y_k are kept in FP64 in the scratch array, so only the stored result is rounded.
template <bool REALCM, int RB, bool C64, int GEN>
__global__ void __launch_bounds__(128) zsolve_kernel(const ZSolveArgs a) {
  const long long plane = (long long)a.nx * a.ny;
  const int ngrp = (a.nrhs + RB - 1) / RB;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= plane * ngrp) return;
  const int grp = (int)(tid / plane);
  const long long pos = tid - (long long)grp * plane;
  const int i = (int)(pos / a.ny), j = (int)(pos - (long long)i * a.ny);
  if (a.skip_i && (a.skip_i[i] | a.skip_j[j])) return;
  const long long rs = plane * a.nz;
  const int r0 = grp * RB;
  const int nr = min(RB, a.nrhs - r0);
  const long long base = r0 * rs + pos;
  // FP64 forward values: the result array itself, or the scratch array for complex64 results
  double2* __restrict__ fw = (C64 ? a.scratch : a.out) + base;
  const double2* __restrict__ P = a.P + pos;
  const double2* __restrict__ Q = a.Q + pos;
  const double2* __restrict__ cm = a.cm;
  const GenThread gt = gen_thread<GEN>(a, i, j);

  double2 y[RB];
#pragma unroll
  for (int q = 0; q < RB; ++q) y[q] = make_double2(0.0, 0.0);
#pragma unroll 2
  for (int k = 0; k < a.nz; ++k) {
    const double2 c = cm[k];
    const double2 pk = P[k * plane];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      if (q < nr) {
        double2 b;
        if constexpr (C64) b = c64_rhs<GEN>(a, gt, base + q * rs + k * plane, r0 + q, k, i, j);
        else b = a.rhs[base + q * rs + k * plane];
        double2 t;
        if (REALCM)
          t = make_double2(fma(-c.x, y[q].x, b.x), fma(-c.x, y[q].y, b.y));
        else
          t = csub_mul(b, c, y[q]);
        y[q] = cmul(t, pk);
        fw[q * rs + k * plane] = y[q];
      }
    }
  }
  if constexpr (C64) {
#pragma unroll
    for (int q = 0; q < RB; ++q)
      if (q < nr) a.out32[base + q * rs + (long long)(a.nz - 1) * plane] = to_c64t(y[q]);
  }
#pragma unroll 2
  for (int k = a.nz - 2; k >= 0; --k) {
    const double2 qk = Q[k * plane];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      if (q < nr) {
        const double2 yk = fw[q * rs + k * plane];
        y[q] = csub_mul(yk, qk, y[q]);
        if constexpr (C64) a.out32[base + q * rs + k * plane] = to_c64t(y[q]);
        else fw[q * rs + k * plane] = y[q];
      }
    }
  }
}

// Few sweeps, long z.  With one thread per sweep and too few sweeps to fill the GPU, the plain
// kernel waits a full memory latency for every z step (its next loads sit behind the current
// step's store).  Here each thread takes z in chunks of 16 steps: all loads of a chunk (P_k,
// the right-hand side, c_k; Q_k and the forward values on the way back) are issued together
// into registers, then the chunk's steps run, with the plain kernel's arithmetic.  (With a
// warp or two per SM sub-partition the step time is then the FP64 pipe's: one warp
// instruction per 64 clocks per sub-partition, 6 of them per forward step with a real c_k,
// 4 per back step.  A form with one multiply-add on the dependency chain,
// y_k = (b_k P_k) - (c_k P_k) y_{k-1}, issues 10 and measured slower.)
constexpr int kZD = 16;

template <bool REALCM, bool C64>
__global__ void __launch_bounds__(128) zsolve_chunk_kernel(const ZSolveArgs a) {
  const long long plane = (long long)a.nx * a.ny;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= plane * a.nrhs) return;
  const int r = (int)(tid / plane);
  const long long pos = tid - (long long)r * plane;
  const int i = (int)(pos / a.ny), j = (int)(pos - (long long)i * a.ny);
  if (a.skip_i && (a.skip_i[i] | a.skip_j[j])) return;
  const long long base = r * plane * a.nz + pos;
  double2* __restrict__ fw = (C64 ? a.scratch : a.out) + base;
  const double2* __restrict__ P = a.P + pos;
  const double2* __restrict__ Q = a.Q + pos;
  const double2* __restrict__ cm = a.cm;
  const int nz = a.nz;
  constexpr int ZD = kZD;
  using RV = typename std::conditional<C64, float2, double2>::type;
  const RV* __restrict__ rhs = C64 ? (const RV*)a.rhs32 : (const RV*)a.rhs;

  double2 y = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < nz; k0 += ZD) {
    // the loads only (a complex64 value is converted where it is used, so that no conversion
    // waits on a load before the next load is issued)
    double2 pk[ZD], ck[ZD];
    RV bk[ZD];
#pragma unroll
    for (int d = 0; d < ZD; ++d) {
      const int k = k0 + d;
      if (k < nz) {
        pk[d] = P[(long long)k * plane];
        bk[d] = rhs[base + (long long)k * plane];
        ck[d] = cm[k];
      }
    }
#pragma unroll
    for (int d = 0; d < ZD; ++d) {
      const int k = k0 + d;
      if (k < nz) {
        const double2 c = ck[d];
        const double2 b = to_c128(bk[d]);
        const double2 t = REALCM ? make_double2(fma(-c.x, y.x, b.x), fma(-c.x, y.y, b.y)) : csub_mul(b, c, y);
        y = cmul(t, pk[d]);
        fw[(long long)k * plane] = y;
      }
    }
  }
  if constexpr (C64) a.out32[base + (long long)(nz - 1) * plane] = to_c64t(y);
  // back substitution over k = nz - 2 .. 0 in chunks of ZD (the last chunk may be short)
  for (int k1 = nz - 2; k1 >= 0; k1 -= ZD) {
    double2 qk[ZD], yk[ZD];
#pragma unroll
    for (int d = 0; d < ZD; ++d) {
      const int k = k1 - d;
      if (k >= 0) {
        qk[d] = Q[(long long)k * plane];
        yk[d] = fw[(long long)k * plane];
      }
    }
#pragma unroll
    for (int d = 0; d < ZD; ++d) {
      const int k = k1 - d;
      if (k >= 0) {
        y = csub_mul(yk[d], qk[d], y);
        if constexpr (C64) a.out32[base + (long long)k * plane] = to_c64t(y);
        else fw[(long long)k * plane] = y;
      }
    }
  }
}

constexpr int RT = 256, REPT = 4;      // right-hand-side kernels: threads, positions per thread

// The right-hand-side kernels below first compute all REPT values of a thread and only
// then store them: the interface arrays are reached through plain struct pointers, so the
// compiler may not move the next position's loads above a store.

// Step 6 boundary term, added in place to the block mode right-hand side:
//   ft[r][k][i][j] += sigma_k (cxl[i] aX[r][k][gxl[i]][j] + cxr[i] aX[r][k][gxr[i]][j]
//                              + cyl[j] aY[r][k][gyl[j]][i] + cyr[j] aY[r][k][gyr[j]][i]).
// REPT positions of a plane per thread, RT * REPT consecutive positions per CTA
// (blockIdx.y = r * nz + k); interface positions are skipped.
// LO: the term is formed in FP32 (mixed path) and added to ft in FP64; FT = float2: ft is
// complex64 (the sum is stored truncated).
template <bool LO, typename FT>
__global__ void __launch_bounds__(RT) boundary_rhs_kernel(const BoundaryArgs a, FT* __restrict__ ft, int rk0) {
  const int rk = rk0 + blockIdx.y;
  const int k = rk % a.nz;
  const int plane = a.nx * a.ny;                           // < 2^31 (checked at plan creation)
  const double s = a.sig ? a.sig[k] : 1.0;
  const double2* __restrict__ axp = a.alphaX + (long long)rk * a.nIx * a.ny;
  const double2* __restrict__ ayp = a.alphaY + (long long)rk * a.nIy * a.nx;
  FT* __restrict__ ftp = ft + (long long)rk * plane;
  double2 val[REPT];
  float2 val32[REPT];
  bool ok[REPT];
#pragma unroll
  for (int e = 0; e < REPT; ++e) {
    const int pos = ((int)blockIdx.x * REPT + e) * RT + (int)threadIdx.x;
    const int i = pos / a.ny, j = pos - i * a.ny;
    ok[e] = pos < plane && !(a.skip_i[i] | a.skip_j[j]);
    if (!ok[e]) continue;
    const int pl = a.gxl[i], pr = a.gxr[i], ql = a.gyl[j], qr = a.gyr[j];
    const double2* ax = axp + j;
    const double2* ay = ayp + i;
    double2 v = to_c128(ftp[pos]);
    if (LO && a.alphaX32) {
      // complex64 interface data and f~: the whole sum in FP32 (one rounding to nearest)
      const float2* ax32 = a.alphaX32 + (long long)rk * a.nIx * a.ny + j;
      const float2* ay32 = a.alphaY32 + (long long)rk * a.nIy * a.nx + i;
      float2 g = make_float2(0.f, 0.f);
      if (pl >= 0) g = cfma32(a.cxl32[i], ax32[(long long)pl * a.ny], g);
      if (pr >= 0) g = cfma32(a.cxr32[i], ax32[(long long)pr * a.ny], g);
      if (ql >= 0) g = cfma32(a.cyl32[j], ay32[(long long)ql * a.nx], g);
      if (qr >= 0) g = cfma32(a.cyr32[j], ay32[(long long)qr * a.nx], g);
      const float2 f32 = to_c64t(ftp[pos]);
      const float s32 = s == 1.0 ? 1.f : f64_to_f32_trunc(s);
      val32[e] = make_float2(fmaf(s32, g.x, f32.x), fmaf(s32, g.y, f32.y));
      continue;
    } else if (LO) {
      float2 g = make_float2(0.f, 0.f);
      if (pl >= 0) g = cfma32(a.cxl32[i], to_c64t(ax[(long long)pl * a.ny]), g);
      if (pr >= 0) g = cfma32(a.cxr32[i], to_c64t(ax[(long long)pr * a.ny]), g);
      if (ql >= 0) g = cfma32(a.cyl32[j], to_c64t(ay[(long long)ql * a.nx]), g);
      if (qr >= 0) g = cfma32(a.cyr32[j], to_c64t(ay[(long long)qr * a.nx]), g);
      const double2 gd = to_c128(g);
      v.x = fma(s, gd.x, v.x);
      v.y = fma(s, gd.y, v.y);
    } else {
      double2 g = make_double2(0.0, 0.0);
      if (a.real_x) {
        if (pl >= 0) g = rfma(a.cxl[i].x, ax[(long long)pl * a.ny], g);
        if (pr >= 0) g = rfma(a.cxr[i].x, ax[(long long)pr * a.ny], g);
      } else {
        if (pl >= 0) g = cfma(a.cxl[i], ax[(long long)pl * a.ny], g);
        if (pr >= 0) g = cfma(a.cxr[i], ax[(long long)pr * a.ny], g);
      }
      if (a.real_y) {
        if (ql >= 0) g = rfma(a.cyl[j].x, ay[(long long)ql * a.nx], g);
        if (qr >= 0) g = rfma(a.cyr[j].x, ay[(long long)qr * a.nx], g);
      } else {
        if (ql >= 0) g = cfma(a.cyl[j], ay[(long long)ql * a.nx], g);
        if (qr >= 0) g = cfma(a.cyr[j], ay[(long long)qr * a.nx], g);
      }
      if (a.sig) {
        v.x = fma(s, g.x, v.x);
        v.y = fma(s, g.y, v.y);
      } else {
        v.x += g.x;
        v.y += g.y;
      }
    }
    val[e] = v;
  }
  if (LO && a.alphaX32) {
#pragma unroll
    for (int e = 0; e < REPT; ++e)
      if (ok[e]) store_f32(ftp + ((int)blockIdx.x * REPT + e) * RT + (int)threadIdx.x, val32[e]);
    return;
  }
#pragma unroll
  for (int e = 0; e < REPT; ++e)
    if (ok[e]) store_c(ftp + ((int)blockIdx.x * REPT + e) * RT + (int)threadIdx.x, val[e]);
}

// Step 5 global right-hand side r~[r][k][l][m] = sum_p Wgx[p][l] aX[r][k][p][m]
//                                              + sum_q Wgy[q][m] bY[r][k][q][l].
// LO: FP32 arithmetic on the FP64 data (mixed path); OT = float2: complex64 output.
template <bool LO, typename OT>
__global__ void __launch_bounds__(RT) global_rhs_kernel(const GlobalRhsArgs a, OT* __restrict__ out,
                                                        int rk0) {
  const int rk = rk0 + blockIdx.y;
  const int plane = a.nx * a.ny;
  const double2* __restrict__ axp = a.aX + (long long)rk * a.nIx * a.ny;
  const double2* __restrict__ byp = a.bY + (long long)rk * a.nIy * a.nx;
  OT* __restrict__ op = out + (long long)rk * plane;
  double2 val[REPT];
  float2 val32[REPT];
#pragma unroll
  for (int e = 0; e < REPT; ++e) {
    const int pos = ((int)blockIdx.x * REPT + e) * RT + (int)threadIdx.x;
    if (pos >= plane) continue;
    const int i = pos / a.ny, j = pos - i * a.ny;
    const double2* ax = axp + j;
    const double2* by = byp + i;
    if (LO && a.aX32) {
      const float2* ax32 = a.aX32 + (long long)rk * a.nIx * a.ny + j;
      const float2* by32 = a.bY32 + (long long)rk * a.nIy * a.nx + i;
      float2 g = make_float2(0.f, 0.f);
      for (int p = 0; p < a.nIx; ++p) g = cfma32(a.WgxI32[(long long)p * a.nx + i], ax32[(long long)p * a.ny], g);
      for (int q = 0; q < a.nIy; ++q) g = cfma32(a.WgyI32[(long long)q * a.ny + j], by32[(long long)q * a.nx], g);
      val32[e] = g;
    } else if (LO) {
      float2 g = make_float2(0.f, 0.f);
      for (int p = 0; p < a.nIx; ++p) g = cfma32(a.WgxI32[(long long)p * a.nx + i], to_c64t(ax[(long long)p * a.ny]), g);
      for (int q = 0; q < a.nIy; ++q) g = cfma32(a.WgyI32[(long long)q * a.ny + j], to_c64t(by[(long long)q * a.nx]), g);
      val[e] = to_c128(g);
    } else {
      double2 b = make_double2(0.0, 0.0);
      if (a.real_x)
        for (int p = 0; p < a.nIx; ++p) b = rfma(a.WgxI[(long long)p * a.nx + i].x, ax[(long long)p * a.ny], b);
      else
        for (int p = 0; p < a.nIx; ++p) b = cfma(a.WgxI[(long long)p * a.nx + i], ax[(long long)p * a.ny], b);
      if (a.real_y)
        for (int q = 0; q < a.nIy; ++q) b = rfma(a.WgyI[(long long)q * a.ny + j].x, by[(long long)q * a.nx], b);
      else
        for (int q = 0; q < a.nIy; ++q) b = cfma(a.WgyI[(long long)q * a.ny + j], by[(long long)q * a.nx], b);
      val[e] = b;
    }
  }
  if (LO && a.aX32) {
#pragma unroll
    for (int e = 0; e < REPT; ++e) {
      const int pos = ((int)blockIdx.x * REPT + e) * RT + (int)threadIdx.x;
      if (pos < plane) store_f32(op + pos, val32[e]);
    }
    return;
  }
#pragma unroll
  for (int e = 0; e < REPT; ++e) {
    const int pos = ((int)blockIdx.x * REPT + e) * RT + (int)threadIdx.x;
    if (pos < plane) store_c(op + pos, val[e]);
  }
}

__global__ void to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) out[t] = to_c64t(in[t]);
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
    // magnitude of the terms summed into the pivot: a pivot at their rounding level is
    // numerically zero (the elimination would amplify rounding errors by 1 / eps)
    double scale = fabs(d.x) + fabs(d.y) + fabs(sk.x) + fabs(sk.y);   // (1-norms bound the moduli)
    d.x += sk.x;
    d.y += sk.y;
    if (k > 0) {
      const double2 c = coff[k];
      const double2 cc = cmul(c, c);
      const double2 ce = cmul(cc, e_prev);
      scale += fabs(ce.x) + fabs(ce.y);
      d = make_double2(d.x - ce.x, d.y - ce.y);
      Q[(long long)(k - 1) * plane + pos] = cmul(c, e_prev);
    }
    const double den = d.x * d.x + d.y * d.y;
    const double mag = sqrt(den);
    if (!(mag > 64.0 * 2.220446049250313e-16 * scale) || !isfinite(mag)) bad = true;
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

template <bool REALCM, bool C64, int GEN>
void launch_sweep(const ZSolveArgs& a, int variant, unsigned grid, cudaStream_t st) {
  const int T = 128;
  if constexpr (GEN == 0) {
    if (variant == 3) zsolve_chunk_kernel<REALCM, C64><<<grid, T, 0, st>>>(a);
    else if (variant == 2) zsolve_kernel<REALCM, 2, C64, 0><<<grid, T, 0, st>>>(a);
    else zsolve_kernel<REALCM, 1, C64, 0><<<grid, T, 0, st>>>(a);
  } else {
    // a sweep that forms its right-hand side takes one RHS per thread
    zsolve_kernel<REALCM, 1, C64, GEN><<<grid, T, 0, st>>>(a);
  }
}

int sweep_variant(const ZSolveArgs& a) {
  const int variant = a.rhs_per_thread;
  if (variant >= 1 && variant <= 3) return variant;
  // automatic: the chunked sweep when the sweeps fill less than 512 threads per SM (the plain
  // kernel then waits a memory latency per z step), else one right-hand side per thread
  // (measured faster on GB300 at the benchmark sizes than two per thread: more independent
  // sweeps in flight beat shared factor loads)
  const long long sweeps = (long long)a.nx * a.ny * a.nrhs;
  return (a.sms > 0 && sweeps < 512LL * a.sms) ? 3 : 1;
}

template <bool REALCM>
void launch_sweep_c(const ZSolveArgs& a, int variant, unsigned grid, cudaStream_t st) {
  if (!a.rhs32) {
    launch_sweep<REALCM, false, 0>(a, variant, grid, st);
  } else if (a.gen.kind == 1) {
    switch (std::max(a.gen.nIx, a.gen.nIy)) {
      case 1: launch_sweep<REALCM, true, 11>(a, variant, grid, st); break;
      case 2: launch_sweep<REALCM, true, 12>(a, variant, grid, st); break;
      case 3: launch_sweep<REALCM, true, 13>(a, variant, grid, st); break;
      default: launch_sweep<REALCM, true, 14>(a, variant, grid, st); break;
    }
  } else if (a.gen.kind == 2) {
    launch_sweep<REALCM, true, 2>(a, variant, grid, st);
  } else {
    launch_sweep<REALCM, true, 0>(a, variant, grid, st);
  }
}

void zsolve(const ZSolveArgs& a, cudaStream_t st) {
  if ((long long)a.nx * a.ny * a.nrhs == 0) return;
  const int T = 128;
  const int variant = sweep_variant(a);
  const int rb = (variant == 2 && a.gen.kind == 0) ? 2 : 1;
  const long long n = (long long)a.nx * a.ny * ((a.nrhs + rb - 1) / rb);
  const unsigned grid = (unsigned)((n + T - 1) / T);
  if (a.real_cm) launch_sweep_c<true>(a, variant, grid, st);
  else launch_sweep_c<false>(a, variant, grid, st);
  count_launch();
}

bool zsolve_forms_rhs(const ZSolveArgs& a) {
  if (sweep_variant(a) == 3) return false;
  if (a.gen.kind == 1) return std::max(a.gen.nIx, a.gen.nIy) >= 1 && std::max(a.gen.nIx, a.gen.nIy) <= kGenMaxIface;
  return a.gen.kind == 2;
}

template <typename FT>
void boundary_rhs_t(const BoundaryArgs& a, FT* ft, cudaStream_t st) {
  const int planes = a.nrhs * a.nz;
  const unsigned gx = (unsigned)(((long long)a.nx * a.ny + RT * REPT - 1) / (RT * REPT));
  for (int rk0 = 0; rk0 < planes; rk0 += 65535) {
    dim3 grid(gx, std::min(65535, planes - rk0));
    if (a.cxl32) boundary_rhs_kernel<true, FT><<<grid, RT, 0, st>>>(a, ft, rk0);
    else boundary_rhs_kernel<false, FT><<<grid, RT, 0, st>>>(a, ft, rk0);
    count_launch();
  }
}
void boundary_rhs(const BoundaryArgs& a, double2* ft, cudaStream_t st) { boundary_rhs_t(a, ft, st); }
void boundary_rhs(const BoundaryArgs& a, float2* ft, cudaStream_t st) { boundary_rhs_t(a, ft, st); }

template <typename OT>
void global_rhs_t(const GlobalRhsArgs& a, OT* out, cudaStream_t st) {
  const int planes = a.nrhs * a.nz;
  const unsigned gx = (unsigned)(((long long)a.nx * a.ny + RT * REPT - 1) / (RT * REPT));
  for (int rk0 = 0; rk0 < planes; rk0 += 65535) {
    dim3 grid(gx, std::min(65535, planes - rk0));
    if (a.WgxI32) global_rhs_kernel<true, OT><<<grid, RT, 0, st>>>(a, out, rk0);
    else global_rhs_kernel<false, OT><<<grid, RT, 0, st>>>(a, out, rk0);
    count_launch();
  }
}
void global_rhs(const GlobalRhsArgs& a, double2* out, cudaStream_t st) { global_rhs_t(a, out, st); }
void global_rhs(const GlobalRhsArgs& a, float2* out, cudaStream_t st) { global_rhs_t(a, out, st); }

void to_c64_copy(const double2* in, float2* out, long long n, cudaStream_t st) {
  if (n <= 0) return;
  to_c64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
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
