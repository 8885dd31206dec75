// Host FP64 mathematics of the ESP planner (see esp_math.h).
//
// Paper references: Eq. pswf (chi = psi_0^c / C0, phi = psi_0^{c1}(2x/(Ph))),
// Eq. hS (Shat(k) = chihat(r_c |k|)/|k|^2), Eq. pk (influence function),
// Eq. errorformula (aliasing), Eq. pswfparameters and Table 2 (parameters).
#include "esp_math.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace espm {

static const double kPi = 3.14159265358979323846;

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged node
    double p1 = 1.0, p2 = 0.0;
    for (int k = 1; k <= n; ++k) {
      double p3 = p2;
      p2 = p1;
      p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
    }
    pp = n * (z * p1 - p2) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

// ----------------------------------------------------------------- Legendre
static void legendre_all(double x, int deg, std::vector<double>& p) {
  p.resize(deg + 1);
  p[0] = 1.0;
  if (deg >= 1) p[1] = x;
  for (int k = 1; k < deg; ++k) p[k + 1] = ((2.0 * k + 1.0) * x * p[k] - k * p[k - 1]) / (k + 1.0);
}

double Pswf::value(double x) const {
  int deg = (int)a.size() - 1;
  // Clenshaw for Legendre: b_k = a_k + alpha_k(x) b_{k+1} + beta_{k+1} b_{k+2}
  double b1 = 0.0, b2 = 0.0;
  for (int k = deg; k >= 0; --k) {
    double alpha = (2.0 * k + 1.0) / (k + 1.0) * x;
    double beta = -(k + 1.0) / (k + 2.0);
    double b0 = a[k] + alpha * b1 + beta * b2;
    b2 = b1;
    b1 = b0;
  }
  return b1;
}

double Pswf::deriv(double x) const {
  int deg = (int)a.size() - 1;
  std::vector<double> p;
  legendre_all(x, deg, p);
  // P'_{k+1} = P'_{k-1} + (2k+1) P_k
  std::vector<double> dp(deg + 1, 0.0);
  if (deg >= 1) dp[1] = 1.0;
  for (int k = 1; k < deg; ++k) dp[k + 1] = dp[k - 1] + (2.0 * k + 1.0) * p[k];
  double s = 0.0;
  for (int k = 0; k <= deg; ++k) s += a[k] * dp[k];
  return s;
}

double Pswf::integral0(double x) const {
  int deg = (int)a.size() - 1;
  std::vector<double> p;
  legendre_all(x, deg + 1, p);
  double s = a[0] * x;
  for (int k = 1; k <= deg; ++k) {
    if (a[k] == 0.0) continue;
    // int_0^x P_k = (P_{k+1}(x) - P_{k-1}(x))/(2k+1) - same at 0 (zero for even k)
    s += a[k] * (p[k + 1] - p[k - 1]) / (2.0 * k + 1.0);
  }
  return s;
}

double Pswf::eigenvalue() const { return 2.0 * a[0] / value(0.0); }

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x.
static int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) ++cnt;
  for (size_t i = 1; i < d.size(); ++i) {
    double prev = (q == 0.0) ? 1e-300 : q;
    q = d[i] - x - e[i - 1] * e[i - 1] / prev;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Solve (T - s I) y = b for the symmetric tridiagonal T (diagonal d,
// off-diagonal e) by Gaussian elimination with partial pivoting; row swaps
// create one extra super-diagonal (u2). A zero pivot is replaced by a tiny
// value: the shifted matrix is meant to be nearly singular (inverse iteration).
static void tridiag_solve(const std::vector<double>& d, const std::vector<double>& e, double s,
                          std::vector<double>& b) {
  const int n = (int)d.size();
  const double tiny = 1e-300;
  std::vector<double> lo(n, 0.0), dg(n), up(n, 0.0), u2(n, 0.0);
  for (int i = 0; i < n; ++i) dg[i] = d[i] - s;
  for (int i = 0; i + 1 < n; ++i) { lo[i] = e[i]; up[i] = e[i]; }   // lo[i] = A(i+1, i)
  for (int i = 0; i + 1 < n; ++i) {
    if (std::fabs(dg[i]) >= std::fabs(lo[i])) {
      double piv = dg[i] != 0.0 ? dg[i] : tiny;
      double f = lo[i] / piv;
      dg[i + 1] -= f * up[i];
      b[i + 1] -= f * b[i];
      u2[i] = 0.0;
    } else {
      // swap rows i and i+1, then eliminate
      double f = dg[i] / lo[i];
      dg[i] = lo[i];
      double t = dg[i + 1];
      dg[i + 1] = up[i] - f * t;
      if (i + 2 < n) {
        u2[i] = up[i + 1];
        up[i + 1] = -f * u2[i];
      }
      up[i] = t;
      double tb = b[i];
      b[i] = b[i + 1];
      b[i + 1] = tb - f * b[i + 1];
    }
  }
  auto piv = [&](int i) { return dg[i] != 0.0 ? dg[i] : tiny; };
  b[n - 1] /= piv(n - 1);
  if (n >= 2) b[n - 2] = (b[n - 2] - up[n - 2] * b[n - 1]) / piv(n - 2);
  for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - up[i] * b[i + 1] - u2[i] * b[i + 2]) / piv(i);
}

Pswf make_pswf(double c) {
  // even-degree normalised-Legendre basis, m terms
  int m = (int)(40 + 1.5 * c);
  std::vector<double> d(m), e(m - 1);
  for (int j = 0; j < m; ++j) {
    double k = 2.0 * j;
    d[j] = k * (k + 1.0) + c * c * (2.0 * k * (k + 1.0) - 1.0) / ((2.0 * k + 3.0) * (2.0 * k - 1.0));
    if (j + 1 < m)
      e[j] = c * c * (k + 2.0) * (k + 1.0) / ((2.0 * k + 3.0) * std::sqrt((2.0 * k + 1.0) * (2.0 * k + 5.0)));
  }
  // Gershgorin bounds, then bisection for the smallest eigenvalue
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < m; ++j) {
    double r = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < m ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (sturm_count(d, e, mid) >= 1) hi = mid; else lo = mid;
    if (hi - lo <= 1e-15 * std::max(1.0, std::fabs(hi))) break;
  }
  double lam = 0.5 * (lo + hi);
  // inverse iteration with a tiny shift below the eigenvalue
  std::vector<double> v(m, 1.0);
  double shift = lam - 1e-10 * std::max(1.0, std::fabs(lam));
  for (int it = 0; it < 4; ++it) {
    tridiag_solve(d, e, shift, v);
    double nrm = 0.0;
    for (double t : v) nrm += t * t;
    nrm = std::sqrt(nrm);
    for (double& t : v) t /= nrm;
  }
  Pswf p;
  p.c = c;
  p.a.assign(2 * m, 0.0);
  for (int j = 0; j < m; ++j) p.a[2 * j] = v[j] * std::sqrt(2.0 * j + 0.5);
  if (p.value(0.0) < 0) for (double& t : p.a) t = -t;
  // trim negligible tail
  double amax = 0.0;
  for (double t : p.a) amax = std::max(amax, std::fabs(t));
  int last = 0;
  for (int k = 0; k < (int)p.a.size(); ++k) if (std::fabs(p.a[k]) > 1e-17 * amax) last = k;
  p.a.resize(last + 1);
  return p;
}

double c_from_tolerance(double eps) {
  double lo = 0.5, hi = 80.0;   // psi_0^c(1) decreases with c
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double v = make_pswf(mid).value(1.0);
    if (v > eps) lo = mid; else hi = mid;
    if (hi - lo < 1e-13) break;
  }
  return 0.5 * (lo + hi);
}

// ------------------------------------------------------------------ splits
static void unit_rule(std::vector<double>& x, std::vector<double>& w, int n) {
  gauss_legendre(n, x, w);
  for (int i = 0; i < n; ++i) { x[i] = 0.5 * (x[i] + 1.0); w[i] *= 0.5; }
}

Split make_pswf_split(double c) {
  Split s;
  s.kind = 0;
  s.c = c;
  s.psi = make_pswf(c);
  s.C0 = s.psi.integral0(1.0);
  unit_rule(s.gx, s.gw, 400);
  s.chi_at.resize(s.gx.size());
  for (size_t i = 0; i < s.gx.size(); ++i) s.chi_at[i] = s.psi.value(s.gx[i]) / s.C0;
  return s;
}

Split make_gauss_split(double alpha) {
  Split s;
  s.kind = 1;
  s.alpha = alpha;
  return s;
}

double Split::chi(double x) const {
  x = std::fabs(x);
  if (kind == 1) return 2.0 * std::sqrt(alpha / kPi) * std::exp(-alpha * x * x);
  if (x > 1.0) return 0.0;
  return psi.value(x) / C0;
}

double Split::dchi(double x) const {
  if (kind == 1) return -2.0 * alpha * x * chi(x);
  return psi.deriv(x) / C0;
}

double Split::one_minus_g(double x) const {
  if (kind == 1) return std::erfc(std::sqrt(alpha) * x);
  if (x >= 1.0) return 0.0;
  return (psi.integral0(1.0) - psi.integral0(x)) / C0;
}

double Split::chihat(double kappa) const {
  if (kind == 1) return std::exp(-kappa * kappa / (4.0 * alpha));
  double s = 0.0;
  for (size_t i = 0; i < gx.size(); ++i) s += gw[i] * chi_at[i] * std::cos(kappa * gx[i]);
  return s;
}

double Split::dchihat(double kappa) const {
  if (kind == 1) return -kappa / (2.0 * alpha) * std::exp(-kappa * kappa / (4.0 * alpha));
  double s = 0.0;
  for (size_t i = 0; i < gx.size(); ++i) s -= gw[i] * gx[i] * chi_at[i] * std::sin(kappa * gx[i]);
  return s;
}

double Split::second_moment() const {
  if (kind == 1) return 1.0 / (2.0 * alpha);
  double s = 0.0;
  for (size_t i = 0; i < gx.size(); ++i) s += gw[i] * gx[i] * gx[i] * chi_at[i];
  return s;
}

Window make_window(double c1, int P) {
  Window w;
  w.c1 = c1;
  w.P = P;
  w.psi = make_pswf(c1);
  unit_rule(w.gx, w.gw, 400);
  w.psi_at.resize(w.gx.size());
  for (size_t i = 0; i < w.gx.size(); ++i) w.psi_at[i] = w.psi.value(w.gx[i]);
  return w;
}

Window make_bspline_window(int P) {
  Window w;
  w.kind = 1;
  w.P = P;
  return w;
}

// Cardinal B-spline M_P(x) on [0, P] by the truncated-power sum.
static double cardinal_bspline(int P, double x) {
  if (!(x > 0.0 && x < P)) return 0.0;
  double s = 0.0, binom = 1.0, fact = 1.0;
  for (int k = 1; k < P; ++k) fact *= k;                  // (P-1)!
  for (int k = 0; k <= P; ++k) {
    const double d = x - k;
    if (d > 0.0) s += ((k & 1) ? -binom : binom) * std::pow(d, P - 1);
    binom = binom * (P - k) / (k + 1);
  }
  return s / fact;
}

double Window::phi(double t) const {
  if (kind == 1) return cardinal_bspline(P, t + 0.5 * P);
  return psi.value(2.0 * t / P);
}

double Window::Phi(double theta) const {
  if (kind == 1) {
    const double h = 0.5 * theta;
    const double sinc = std::fabs(h) > 1e-12 ? std::sin(h) / h : 1.0;
    return std::pow(sinc, P);
  }
  // int_{-P/2}^{P/2} psi(2t/P) cos(theta t) dt = P int_0^1 psi(x) cos(theta P x / 2) dx
  double s = 0.0;
  for (size_t i = 0; i < gx.size(); ++i) s += gw[i] * psi_at[i] * std::cos(0.5 * theta * P * gx[i]);
  return P * s;
}

double alias_relative(const Split& s, const Window& w, int n_f, double L, double r_c) {
  int h = n_f / 2;
  int mmax = 3 * h * h;
  std::vector<double> base(mmax + 1, 0.0);
  for (int m = 1; m <= mmax; ++m)
    base[m] = std::fabs(s.chihat(2.0 * kPi * r_c * std::sqrt((double)m) / L)) / m;
  double num = 0.0, den = 0.0;
  for (int kx = -h; kx < h; ++kx) {
    double th = 2.0 * kPi * kx / n_f;
    double ratio = std::fabs(w.Phi(th + 2.0 * kPi) / w.Phi(th));
    double row = 0.0;
    for (int ky = -h; ky < h; ++ky)
      for (int kz = -h; kz < h; ++kz) row += base[kx * kx + ky * ky + kz * kz];
    num += ratio * row;
    den += row;
  }
  return 6.0 * num / den;
}

int stencil_width(double eps) {
  // Table 2: 1e-3 -> 5, 5e-4 -> 5, 1e-4 -> 6, 5e-5 -> 7, 1e-5 -> 8
  const double tol[5] = {1e-3, 5e-4, 1e-4, 5e-5, 1e-5};
  const int P[5] = {5, 5, 6, 7, 8};
  for (int i = 0; i < 5; ++i) if (eps >= tol[i] * (1 - 1e-12)) return P[i];
  return (int)std::ceil(std::log10(1.0 / eps)) + 3;
}

double default_grid_ratio(double eps) {
  // Table 2, last row: R_default = 5.78, 7.71, 14.32, 22.42, 54.57 at
  // eps = 1e-3, 5e-4, 1e-4, 5e-5, 1e-5; (log eps, log R) interpolated
  // linearly, extrapolated along the nearest segment; per axis R^(1/3)
  const double tol[5] = {1e-5, 5e-5, 1e-4, 5e-4, 1e-3};
  const double R[5] = {54.57, 22.42, 14.32, 7.71, 5.78};
  const double lx = std::log(eps);
  int k = 0;
  while (k < 3 && lx > std::log(tol[k + 1])) ++k;
  const double x0 = std::log(tol[k]), x1 = std::log(tol[k + 1]);
  const double y0 = std::log(R[k]), y1 = std::log(R[k + 1]);
  return std::exp((y0 + (y1 - y0) * (lx - x0) / (x1 - x0)) / 3.0);
}

bool is_smooth(int n) {
  if (n <= 0) return false;
  for (int p : {2, 3, 5, 7}) while (n % p == 0) n /= p;
  return n == 1;
}

int round_grid(double n) {
  int m = std::max(2, (int)std::ceil(n - 1e-9));
  if (m % 2) ++m;
  while (!is_smooth(m)) m += 2;
  return m;
}

}  // namespace espm
