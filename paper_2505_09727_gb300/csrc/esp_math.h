// Host FP64 mathematics of the ESP planner: prolate spheroidal wave functions,
// splitting functions, SI-kernel transforms, the aliasing estimate, and the
// polynomial fits the kernels evaluate. One-time work per plan.
#pragma once
#include <cstdint>
#include <vector>

namespace espm {

// Gauss-Legendre nodes/weights on [-1,1] (Newton on the three-term recurrence).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// psi_0^c as a Legendre series sum a_k P_k(x) (even k), L2-normalised on
// [-1,1] with psi(0) > 0. Built from the prolate differential operator, whose
// matrix in the normalised Legendre basis is symmetric tridiagonal; psi_0^c
// is the eigenvector of its smallest eigenvalue (Sturm bisection + inverse
// iteration).
struct Pswf {
  double c = 0;
  std::vector<double> a;     // plain-Legendre coefficients, index = degree
  double value(double x) const;
  double deriv(double x) const;
  double integral0(double x) const;   // int_0^x psi
  double eigenvalue() const;          // lambda of F_c[psi] = lambda psi
};
Pswf make_pswf(double c);

// c with psi_0^c(1) = eps (bisection).
double c_from_tolerance(double eps);

// Splitting kernel chi on [0,1] (PSWF: psi/C0, C0 = int_0^1 psi, truncated at
// 1) or the Gaussian 2 sqrt(alpha/pi) exp(-alpha x^2).
struct Split {
  int kind = 0;              // 0 = PSWF, 1 = Gauss
  double c = 0, alpha = 0, C0 = 1;
  Pswf psi;
  std::vector<double> gx, gw, chi_at;   // 0..1 Gauss-Legendre rule and chi there
  double chi(double x) const;
  double one_minus_g(double x) const;   // int_x^1 chi (PSWF) or erfc(sqrt(a) x)
  double dchi(double x) const;          // chi'(x) for 0 <= x <= 1
  double chihat(double kappa) const;    // int_0^inf chi(x) cos(kappa x) dx
  double dchihat(double kappa) const;   // d chihat / d kappa
  double chi0() const { return chi(0.0); }
  double second_moment() const;         // int_0^inf x^2 chi
};
Split make_pswf_split(double c);
Split make_gauss_split(double alpha);

// SI kernel phi(t) in grid units t and its transform.
// kind 0: PSWF window psi_0^{c1}(2t/P); kind 1: centred cardinal B-spline of
// order P (piecewise polynomial of degree P-1, transform (sin(x/2)/(x/2))^P).
struct Window {
  int kind = 0;
  double c1 = 0;
  int P = 0;
  Pswf psi;
  std::vector<double> gx, gw, psi_at;
  double phi(double t) const;            // analytic on the support (no support cut for kind 0)
  double Phi(double theta) const;        // int phi(t) cos(theta t) dt over |t|<=P/2
};
Window make_window(double c1, int P);
Window make_bspline_window(int P);

// Relative aliasing estimate (Eq. errorformula divided by the same sum
// without the alias ratio).
double alias_relative(const Split& s, const Window& w, int n_f, double L, double r_c);

// Table 2 stencil width, smooth even grid sizes.
int stencil_width(double eps);
// Table 2's R_default^(1/3): per-axis grid ratio of the default PME
// (Gaussian split, B-spline order 5) to ESP at the same error.
double default_grid_ratio(double eps);
bool is_smooth(int n);
int round_grid(double n);

}  // namespace espm
