// Generalised eigenpairs of a complex-symmetric tridiagonal pencil (K, M), M diagonal.
//
// The x/y transforms of Sec. 2 need, per block and for the whole axis, the
// generalised eigenpairs A_d W = M_d W Lambda with W = 0 on the block boundary
// (display after Eq. (fdmtrprj); global pairs before Eq. (fdmtrprjfrerr)).
// With complex (PML) steps K and M are complex symmetric, not Hermitian, so
// the pairs are computed with complex-orthogonal similarity transforms:
//
//   T = M^{-1/2} K M^{-1/2}  (principal square roots; T complex symmetric tridiagonal)
//   T = Z Lambda Z^T with Z^T Z = I, by the implicit QL iteration with a
//   Wilkinson shift, each step a chain of plane rotations R = [[c, -s], [s, c]]
//   with c^2 + s^2 = 1 (complex c, s) that chases the bulge from the bottom of
//   the active block to its top (Cullum & Willoughby, complex symmetric QL);
//   W = M^{-1/2} Z, so that W^T M W = Z^T Z = I and K W = M W Lambda.
//
// The routine reports failure (no convergence, a rotation with c^2 + s^2 = 0)
// instead of returning inaccurate pairs; the caller also checks both
// identities on the result.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "hz_internal.h"

namespace hz {

namespace {

// One implicit QL sweep on the unreduced block [l, m] of (d, e) with shift mu;
// Z (n x n, row-major) accumulates the rotations.  Returns false on breakdown.
bool ql_sweep(int n, int l, int m, cd mu, std::vector<cd>& d, std::vector<cd>& e, std::vector<cd>& Z) {
  // First rotation: zero the (m-1, m) entry of (T - mu I) from the bottom.
  cd x = d[m] - mu;
  cd y = e[m - 1];
  for (int p = m - 1; p >= l; --p) {
    const int q = p + 1;
    cd rho = std::sqrt(x * x + y * y);
    const double scale = std::abs(x) + std::abs(y);
    if (scale == 0.0) return false;
    if (std::abs(rho) <= 1e-10 * scale) return false;       // isotropic pair: c^2 + s^2 = 0
    const cd c = x / rho, s = y / rho;
    if (p < m - 1) e[q] = rho;                               // bulge at (p, q+1) annihilated
    const cd dp = d[p], dq = d[q], ep = e[p];
    const cd cc = c * c, ss = s * s, cs = c * s;
    d[p] = cc * dp - 2.0 * cs * ep + ss * dq;
    d[q] = ss * dp + 2.0 * cs * ep + cc * dq;
    e[p] = cs * (dp - dq) + (cc - ss) * ep;
    if (p > l) {                                             // new bulge at (p-1, p+1)
      const cd bulge = s * e[p - 1];
      e[p - 1] = c * e[p - 1];
      x = e[p];
      y = bulge;
    }
    for (int k = 0; k < n; ++k) {                            // Z <- Z R^T on columns p, q
      const cd zp = Z[(size_t)k * n + p], zq = Z[(size_t)k * n + q];
      Z[(size_t)k * n + p] = c * zp - s * zq;
      Z[(size_t)k * n + q] = s * zp + c * zq;
    }
  }
  return true;
}

}  // namespace

bool tridiag_eig(int n, const cd* kd, const cd* ko, const cd* m, std::vector<cd>& lam,
                 std::vector<cd>& W, double* eig_residual) {
  lam.assign(n, cd(0));
  W.assign((size_t)n * n, cd(0));
  if (n <= 0) return false;
  std::vector<cd> sm(n), d(n), e(std::max(n, 1), cd(0));
  for (int i = 0; i < n; ++i) {
    sm[i] = std::sqrt(m[i]);
    d[i] = kd[i] / m[i];
  }
  for (int i = 0; i + 1 < n; ++i) e[i] = ko[i] / (sm[i] * sm[i + 1]);
  std::vector<cd> Z((size_t)n * n, cd(0));
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;

  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int mm = l;
      for (; mm < n - 1; ++mm) {
        const double dd = std::abs(d[mm]) + std::abs(d[mm + 1]);
        if (std::abs(e[mm]) <= eps * dd) break;
      }
      if (mm == l) break;
      if (++iter > 200) return false;
      if (mm < n - 1) e[mm] = 0.0;                                  // exact split below the block
      // Wilkinson shift: eigenvalue of the leading 2x2 of the block closest to d[l].
      const cd a = d[l], b = d[l + 1], c = e[l];
      const cd half = 0.5 * (a - b);
      const cd disc = std::sqrt(half * half + c * c);
      const cd mu1 = 0.5 * (a + b) + disc, mu2 = 0.5 * (a + b) - disc;
      cd mu = (std::abs(mu1 - a) <= std::abs(mu2 - a)) ? mu1 : mu2;
      if (iter % 20 == 0) mu += 1e-3 * std::abs(c) * cd(1.0, 0.5);   // exceptional shift
      if (!ql_sweep(n, l, mm, mu, d, e, Z)) return false;
    }
  }
  // Sort by (Re, Im) of lambda for reproducible tables; W = M^{-1/2} Z.
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (d[a].real() != d[b].real()) return d[a].real() < d[b].real();
    return d[a].imag() < d[b].imag();
  });
  for (int col = 0; col < n; ++col) {
    const int src = order[col];
    lam[col] = d[src];
    for (int i = 0; i < n; ++i) W[(size_t)i * n + col] = Z[(size_t)i * n + src] / sm[i];
  }
  const double res = eig_check(n, kd, ko, m, lam, W);
  if (eig_residual) *eig_residual = res;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(lam[i].real()) || !std::isfinite(lam[i].imag())) return false;
  return true;
}

// max(||K W - M W Lambda||_F / (||K||_F ||W||_F), max |W^T M W - I|).
double eig_check(int n, const cd* kd, const cd* ko, const cd* m, const std::vector<cd>& lam,
                 const std::vector<cd>& W) {
  double rk = 0, nk = 0, nw = 0, orth = 0;
  for (int i = 0; i < n; ++i) {
    nk += std::norm(kd[i]) + (i + 1 < n ? 2.0 * std::norm(ko[i]) : 0.0);
    for (int col = 0; col < n; ++col) {
      cd kw = kd[i] * W[(size_t)i * n + col];
      if (i > 0) kw += ko[i - 1] * W[(size_t)(i - 1) * n + col];
      if (i + 1 < n) kw += ko[i] * W[(size_t)(i + 1) * n + col];
      rk += std::norm(kw - m[i] * W[(size_t)i * n + col] * lam[col]);
      nw += std::norm(W[(size_t)i * n + col]);
    }
  }
  for (int a = 0; a < n; ++a)
    for (int b = a; b < n; ++b) {
      cd g = 0;
      for (int i = 0; i < n; ++i) g += W[(size_t)i * n + a] * m[i] * W[(size_t)i * n + b];
      const double dev = std::abs(g - (a == b ? cd(1.0) : cd(0.0)));
      orth = std::max(orth, dev);
    }
  return std::max(std::sqrt(rk) / (std::sqrt(nk) * std::sqrt(nw)), orth);
}

// Uniform real block (n nodes, all n + 1 steps equal to h > 0): K = tridiag(-1, 2, -1) / h and
// M = h I have the discrete sine eigenpairs
//   lambda_m = (4 / h^2) sin^2(m pi / (2 (n + 1))),  w_m[i] = sqrt(2 / ((n + 1) h)) sin((i + 1) m pi / (n + 1)),
// m = 1..n, with W^T M W = I.  w_m is symmetric under i -> n - 1 - i for odd m and
// antisymmetric for even m; the columns hold the odd m first (column l < (n + 1) / 2 is
// m = 2 l + 1), then the even m, which the row transforms use to halve their work.
bool sine_eig(int n, double h, const cd* kd, const cd* ko, const cd* m, std::vector<cd>& lam,
              std::vector<cd>& W, double* eig_residual) {
  if (n < 1 || !(h > 0.0)) return false;
  const double pi = 3.14159265358979323846;
  const double L = n + 1.0;
  const double c = std::sqrt(2.0 / (L * h));
  lam.assign(n, cd(0));
  W.assign((size_t)n * n, cd(0));
  const int ns = (n + 1) / 2;
  for (int col = 0; col < n; ++col) {
    const int mm = col < ns ? 2 * col + 1 : 2 * (col - ns) + 2;
    const double sn = std::sin(mm * pi / (2.0 * L));
    lam[col] = cd(4.0 / (h * h) * sn * sn, 0.0);
    for (int i = 0; i < n; ++i) {
      const long long arg = (long long)(i + 1) * mm % (2 * (n + 1));   // exact reduction mod 2 pi
      W[(size_t)i * n + col] = cd(c * std::sin((double)arg * pi / L), 0.0);
    }
  }
  const double res = eig_check(n, kd, ko, m, lam, W);
  if (eig_residual) *eig_residual = res;
  return true;
}

}  // namespace hz
