// Host-side special functions and small linear algebra for the setup phase.
#include <cmath>
#include <vector>
#include "prd_internal.h"

namespace prd {

// Faddeeva function by Weideman's rational expansion (J.A.C. Weideman, SIAM
// J. Numer. Anal. 31 (1994) 1497): with Z = (L + i z)/(L - i z),
//   w(z) = 2 sum_{k>=1} a_k Z^{k-1} / (L - i z)^2 + 1/(sqrt(pi)(L - i z)),
// a_k the Fourier coefficients of exp(-t^2)(L^2 + t^2) under t = L tan(th/2).
void weideman_coeffs(int n, double* a_out, double* L_out) {
  const double L = std::sqrt((double)n) / std::pow(2.0, 0.25);
  const int M = 8 * n;                 // trapezoidal points on (-pi, pi]
  std::vector<double> psi(2 * M);
  for (int j = 0; j < 2 * M; ++j) {
    const int kk = j - M + 1;          // -M+1 .. M
    const double th = kPi * kk / M;
    if (kk == M) { psi[j] = 0.0; continue; }
    const double t = L * std::tan(0.5 * th);
    psi[j] = std::exp(-t * t) * (L * L + t * t);
  }
  for (int k = 1; k <= n; ++k) {
    double s = 0.0;
    for (int j = 0; j < 2 * M; ++j) {
      const int kk = j - M + 1;
      s += psi[j] * std::cos(k * kPi * kk / M);
    }
    a_out[k - 1] = s / (2.0 * M);
  }
  *L_out = L;
}

namespace {
struct WCoef {
  double a[kWeidemanN64];
  double L;
  WCoef() { weideman_coeffs(kWeidemanN64, a, &L); }
};
const WCoef& wcoef() {
  static WCoef w;
  return w;
}
}  // namespace

cplx faddeeva_host(cplx z) {
  const WCoef& w = wcoef();
  const cplx iz(-z.imag(), z.real());
  const cplx d = w.L - iz;
  const cplx Z = (w.L + iz) / d;
  cplx p = 0.0;
  for (int k = kWeidemanN64 - 1; k >= 0; --k) p = p * Z + w.a[k];
  return 2.0 * p / (d * d) + 1.0 / (kSqrtPi * d);
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1], Newton on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[n - 1 - i] = t;   // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Natural cubic spline (zero end second derivatives): Q maps node values to
// second derivatives M = Q y.  Rows 0 and n-1 are zero.  Row-major n x n.
void natural_spline_Q(const double* u, int n, double* Q) {
  for (int i = 0; i < n * n; ++i) Q[i] = 0.0;
  if (n <= 2) return;
  const int m = n - 2;
  std::vector<double> h(n - 1);
  for (int i = 0; i < n - 1; ++i) h[i] = u[i + 1] - u[i];
  // tridiagonal (m x m): sub = h[i-1], diag = 2(h[i-1]+h[i]), sup = h[i]  (i = 1..n-2)
  std::vector<double> cp(m), dn(m);
  for (int r = 0; r < m; ++r) {
    const int i = r + 1;
    const double sub = (r > 0) ? h[i - 1] : 0.0;
    const double dg = 2.0 * (h[i - 1] + h[i]);
    const double den = dg - sub * (r > 0 ? cp[r - 1] : 0.0);
    dn[r] = den;
    cp[r] = (r < m - 1) ? h[i] / den : 0.0;
  }
  std::vector<double> rhs(m), sol(m);
  for (int col = 0; col < n; ++col) {
    for (int r = 0; r < m; ++r) {
      const int i = r + 1;
      double v = 0.0;
      if (col == i + 1) v += 6.0 / h[i];
      if (col == i) v -= 6.0 / h[i] + 6.0 / h[i - 1];
      if (col == i - 1) v += 6.0 / h[i - 1];
      rhs[r] = v;
    }
    // forward sweep
    for (int r = 0; r < m; ++r) {
      const int i = r + 1;
      const double sub = (r > 0) ? h[i - 1] : 0.0;
      rhs[r] = (rhs[r] - sub * (r > 0 ? rhs[r - 1] : 0.0)) / dn[r];
    }
    for (int r = m - 1; r >= 0; --r) sol[r] = rhs[r] - (r < m - 1 ? cp[r] * sol[r + 1] : 0.0);
    for (int r = 0; r < m; ++r) Q[(r + 1) * n + col] = sol[r];
  }
}

}  // namespace prd
