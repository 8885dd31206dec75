// Host planning of one system (see esp_plan.h).
//
// Parameter rules (paper, Methods):
//  * c from psi_0^c(1) = eps (Eq. pswfparameters), P from Table 2;
//  * n_f starts at ceil(c L / (pi r_c)) (PSWF, Eq. pswfparameters) or
//    2 ceil(ln(1/eps) L / (pi r_c)) (Gaussian, Eq. cemparameters), rounded to
//    an even FFT-friendly size;
//  * the SI-kernel shape c1 is the one of c1/c in {1.10, 1.15, ..., 1.40} that
//    minimises the relative aliasing estimate (Eq. errorformula), and n_f is
//    raised until that minimum is at most eps/2 (the paper lets n_f grow until
//    the estimate is of the order of the tolerance);
//  * r_c, when not given, minimises a GPU cost model of the local and
//    spectral parts (the paper leaves r_c free to balance the two costs).
#include "esp_plan.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

namespace espe {

static const double kPi = 3.14159265358979323846;

// The PSWF solves depend only on (eps), (c) and (c1, P); batches plan many
// systems with the same values, so the results are kept per process.
static std::mutex g_cache_mu;

static double cached_c(double eps) {
  static std::map<double, double> cache;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = cache.find(eps);
    if (it != cache.end()) return it->second;
  }
  const double c = espm::c_from_tolerance(eps);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  cache[eps] = c;
  return c;
}

static espm::Split cached_pswf_split(double c) {
  static std::map<double, espm::Split> cache;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = cache.find(c);
    if (it != cache.end()) return it->second;
  }
  espm::Split s = espm::make_pswf_split(c);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (cache.size() > 64) cache.clear();
  cache[c] = s;
  return s;
}

static espm::Window cached_window(double c1, int P) {
  static std::map<std::pair<double, int>, espm::Window> cache;
  const auto key = std::make_pair(c1, P);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  espm::Window w = espm::make_window(c1, P);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (cache.size() > 256) cache.clear();
  cache[key] = w;
  return w;
}

// chihat(r_c xi_m) at the radial modes xi_m = 2 pi sqrt(m) / L of a cube
// (m = |k|^2), evaluated once per m and shared by the aliasing estimates of
// every grid size tried and the influence table.
class RadialChihat {
 public:
  RadialChihat(const espm::Split& s, double L, double r_c) : s_(s), L_(L), r_c_(r_c) {}
  double operator()(int m) {
    while ((int)v_.size() <= m) {
      const double xi = 2.0 * kPi * std::sqrt((double)v_.size()) / L_;
      v_.push_back(s_.chihat(r_c_ * xi));
    }
    return v_[m];
  }

 private:
  const espm::Split& s_;
  double L_, r_c_;
  std::vector<double> v_;
};

// Sum over ky, kz of |chihat(2 pi r_c |k| / L)| / |k|^2 for each kx in I.
static std::vector<double> alias_rows(RadialChihat& chi, int n_f) {
  const int h = n_f / 2;
  const int mmax = 3 * h * h;
  std::vector<double> base(mmax + 1, 0.0);
  chi(mmax);
  for (int m = 1; m <= mmax; ++m) base[m] = std::fabs(chi(m)) / m;
  // rows[kx] = sum_{ky,kz} base[kx^2 + ky^2 + kz^2] = sum_s n(s) base[kx^2 + s]
  // with n(s) the number of (ky, kz) in [-h, h)^2 with ky^2 + kz^2 = s (most
  // s are no sum of two squares), and rows even in kx
  std::vector<int> count(2 * h * h + 1, 0);
  for (int ky = -h; ky < h; ++ky)
    for (int kz = -h; kz < h; ++kz) ++count[ky * ky + kz * kz];
  std::vector<int> sums;
  std::vector<double> mult;
  for (int v = 0; v <= 2 * h * h; ++v)
    if (count[v]) {
      sums.push_back(v);
      mult.push_back((double)count[v]);
    }
  std::vector<double> rows(n_f, 0.0);
  for (int k = 0; k <= h; ++k) {
    const double* b = base.data() + k * k;
    double r = 0.0;
    for (size_t i = 0; i < sums.size(); ++i) r += mult[i] * b[sums[i]];
    if (k < h) rows[h + k] = r;        // kx = k
    rows[h - k] = r;                   // kx = -k (k = h: the -n_f/2 row)
  }
  return rows;
}

static double alias_from_rows(const std::vector<double>& rows, const espm::Window& w, int n_f) {
  const int h = n_f / 2;
  double num = 0.0, den = 0.0;
  for (int kx = -h; kx < h; ++kx) {
    const double th = 2.0 * kPi * kx / n_f;
    const double ratio = std::fabs(w.Phi(th + 2.0 * kPi) / w.Phi(th));
    num += ratio * rows[kx + h];
    den += rows[kx + h];
  }
  return 6.0 * num / den;
}

// GPU cost model (seconds) used only to pick r_c when the caller does not.
static double model_cost(double L, long long N, int P, double c, double r_c, int kernel, double tol) {
  const double rho = (double)N / (L * L * L);
  const double nmin = kernel == ESP_KERNEL_PSWF ? c * L / (kPi * r_c)
                                                : 2.0 * std::ceil(std::log(1.0 / tol) * L / (kPi * r_c));
  const int n_f = espm::round_grid(nmin);
  if (n_f > 1024) return 1e30;
  const int n_c = std::max(1, (int)std::floor(2.0 * L / r_c));
  const double cell = L / n_c;
  const double cand = n_c >= 5 ? 125.0 * cell * cell * cell * rho : (double)N;
  const double nf3 = (double)n_f * n_f * n_f;
  const double t_near = 2.5e-13 * (double)N * cand;
  const double t_sg = 1.5e-13 * (double)N * P * P * P;
  const double t_fft = 2.0 * 1.0e-12 * nf3 * std::log2(std::max(8.0, nf3)) + 2.0e-5;
  return t_near + t_sg + t_fft;
}

// Chebyshev interpolation of f on y in [-1,1] at degree `deg`, converted to
// monomial coefficients in y (out[k] multiplies y^k); returns the max error of
// the monomial form on a fine sample.
template <class F>
static double fit(F f, int deg, std::vector<double>& out) {
  const int n = deg + 1;
  const double pi = kPi;
  std::vector<double> fv(n), cheb(n, 0.0);
  for (int j = 0; j < n; ++j) fv[j] = f(std::cos(pi * (j + 0.5) / n));
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += fv[j] * std::cos(pi * k * (j + 0.5) / n);
    cheb[k] = (k == 0 ? 1.0 : 2.0) * s / n;
  }
  out.assign(n, 0.0);
  std::vector<double> tprev(n, 0.0), tcur(n, 0.0), tnext(n, 0.0);
  tprev[0] = 1.0;
  if (n > 1) tcur[1] = 1.0;
  out[0] += cheb[0];
  if (n > 1) out[1] += cheb[1];
  for (int k = 2; k < n; ++k) {
    std::fill(tnext.begin(), tnext.end(), 0.0);
    for (int i = 0; i + 1 < n; ++i) tnext[i + 1] += 2.0 * tcur[i];
    for (int i = 0; i < n; ++i) tnext[i] -= tprev[i];
    for (int i = 0; i < n; ++i) out[i] += cheb[k] * tnext[i];
    tprev.swap(tcur);
    tcur.swap(tnext);
  }
  double err = 0.0;
  for (int i = 0; i <= 1000; ++i) {
    const double y = -1.0 + 2.0 * i / 1000.0;
    double v = 0.0;
    for (int k = n - 1; k >= 0; --k) v = v * y + out[k];
    err = std::max(err, std::fabs(v - f(y)));
  }
  return err;
}

// Piecewise SI-kernel polynomials: piece a of phi on t in [a - P/2 + 1 ... ]
// as a polynomial in y = 2 delta - 1, both precisions.
struct SiTables {
  espk::SICoef<float> si32{};
  espk::SICoef<double> si64{};
  double err32 = 0, err64 = 0;
};

static SiTables make_si_tables(const espm::Window& win, int P) {
  SiTables t;
  std::vector<double> co;
  for (int a = 0; a < P; ++a) {
    auto fa = [&](double y) { return win.phi(0.5 * (y + 1.0) + 0.5 * P - 1.0 - a); };
    t.err32 = std::max(t.err32, fit(fa, espk::Deg<float>::si - 1, co));
    for (int k = 0; k < espk::Deg<float>::si; ++k) t.si32.c[a][k] = (float)co[k];
    t.err64 = std::max(t.err64, fit(fa, espk::Deg<double>::si - 1, co));
    for (int k = 0; k < espk::Deg<double>::si; ++k) t.si64.c[a][k] = co[k];
  }
  return t;
}

static const SiTables& si_tables(const espm::Window& win, int P) {
  static std::map<std::pair<double, int>, SiTables> cache;
  const auto key = std::make_pair(win.c1, P);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  SiTables t = make_si_tables(win, P);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  return cache.emplace(key, t).first->second;
}

// Local-part polynomials in y = 2s - 1, s = (r/r_c)^2:
// H(s) = g(x)/x and K(s) = (x chi(x) - g(x))/x^3, x = sqrt(s), with K in the
// cancellation-free form K = (1/x) int_0^1 u chi'(x u) du.
struct NearTables {
  espk::NearCoef<float> nc32{};
  espk::NearCoef<double> nc64{};
  int terms32 = 0;
  double err32 = 0, err64 = 0;
};

static NearTables make_near_tables(const espm::Split& split, double tol) {
  NearTables t;
  std::vector<double> gq_x, gq_w, co;
  espm::gauss_legendre(48, gq_x, gq_w);
  for (size_t i = 0; i < gq_x.size(); ++i) { gq_x[i] = 0.5 * (gq_x[i] + 1.0); gq_w[i] *= 0.5; }
  auto g_of = [&](double x) {
    return split.kind == 1 ? std::erf(std::sqrt(split.alpha) * x) : split.psi.integral0(x) / split.C0;
  };
  auto fh = [&](double y) {
    const double x = std::sqrt(std::max(0.0, 0.5 * (y + 1.0)));
    return x > 1e-12 ? g_of(x) / x : split.chi0();
  };
  auto fk = [&](double y) {
    const double x = std::max(1e-9, std::sqrt(std::max(0.0, 0.5 * (y + 1.0))));
    double acc = 0.0;
    for (size_t i = 0; i < gq_x.size(); ++i) acc += gq_w[i] * gq_x[i] * split.dchi(x * gq_x[i]);
    return acc / x;
  };
  // FP32: the fewest of 8, 9, 10 or 12 terms whose fit error is 100x below
  // the tolerance
  const double scale = std::max(std::fabs(fh(-1.0)), std::fabs(fk(1.0)));
  for (int terms : {8, 9, 10, espk::Deg<float>::nr}) {
    std::vector<double> ch, ck;
    const double e1 = fit(fh, terms - 1, ch);
    const double e2 = fit(fk, terms - 1, ck);
    t.terms32 = terms;
    t.err32 = std::max(e1, e2);
    for (int k = 0; k < espk::Deg<float>::nr; ++k) {
      t.nc32.h[k] = k < terms ? (float)ch[k] : 0.0f;
      t.nc32.k[k] = k < terms ? (float)ck[k] : 0.0f;
    }
    if (t.err32 <= 0.01 * tol * std::max(1.0, scale)) break;
  }
  const double e3 = fit(fh, espk::Deg<double>::nr - 1, co);
  for (int k = 0; k < espk::Deg<double>::nr; ++k) t.nc64.h[k] = co[k];
  const double e4 = fit(fk, espk::Deg<double>::nr - 1, co);
  for (int k = 0; k < espk::Deg<double>::nr; ++k) t.nc64.k[k] = co[k];
  t.err64 = std::max(e3, e4);
  return t;
}

static const NearTables& near_tables(const espm::Split& split, double tol) {
  static std::map<std::pair<std::pair<int, double>, double>, NearTables> cache;
  const auto key = std::make_pair(std::make_pair(split.kind, split.kind == 1 ? split.alpha : split.c), tol);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  NearTables t = make_near_tables(split, tol);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  return cache.emplace(key, t).first->second;
}

static int tile_edge(const espk::SysDesc& d, int P, int precision) {
  int T = 0;
  for (int cb = 0; cb < d.nb; ++cb) {
    int t;
    if (precision == ESP_FP32) {
      t = espk::tile_last_fixed((cb + 1) * d.bc, d.n_c, d.n_f, P) -
          espk::tile_origin_fixed(cb * d.bc, d.n_c, d.n_f, P) + P;
    } else {
      double dl;
      const int lo = espk::stencil_origin_f64((double)(cb * d.bc) * d.L / d.n_c, d.L, d.n_f, P, dl);
      const int hi = espk::stencil_origin_f64((double)((cb + 1) * d.bc) * d.L / d.n_c, d.L, d.n_f, P, dl);
      t = hi - lo + P + 2;
    }
    T = std::max(T, t);
  }
  return T;
}

// Cell count n_c <= nc_max (a multiple of the brick edge bc) and the tile edge
// T of the spread and gather bricks. A brick is bc^3 cells; the choice prefers
// a brick edge near 6.5 grid points (measured best for the spread and gather
// tiles) among shapes that keep at least 90% of the finest admissible cell
// count. L only feeds the FP64 tile bound (FP64 coordinates are Cartesian).
static esp_status choose_bricks(int n_f, int nc_max, double L, int P, const esp_plan_opts& o, int& n_c, int& bc,
                                int& T, std::string& msg) {
  const int prec = o.precision;
  n_c = bc = T = 0;
  double best_score = -1e300;
  const size_t rb = prec == ESP_FP32 ? 4 : 8;
  for (int b = 1; b <= 8; ++b) {
    if (o.brick_cells > 0 && b != o.brick_cells) continue;
    const int nc = (nc_max / b) * b;
    if (nc < b || nc == 0) continue;
    espk::SysDesc d{};
    d.n_f = n_f; d.n_c = nc; d.bc = b; d.nb = nc / b;
    d.L = L; d.inv_h = n_f / L;
    const int t = tile_edge(d, P, prec);
    int tpy = 0, tpz = 0;
    espk::tile_pitches(t, P, tpy, tpz);
    const size_t tiles = o.diff == ESP_DIFF_IK ? 4 : 1;      // the ik gather holds four tiles
    if ((size_t)tpz * t * rb * tiles > 200 * 1024) continue;
    const double edge = (double)b * n_f / nc;            // brick edge in grid points
    const double keep = (double)nc / nc_max;
    double score = -std::fabs(std::log(edge / 6.5));
    if (keep < 0.9) score -= 10.0 + (1.0 - keep) * 10.0;
    if (score > best_score) { best_score = score; n_c = nc; bc = b; T = t; }
  }
  if (o.brick_cells > 0 && n_c == 0) {
    // requested brick does not divide any usable cell count: use single-cell bricks
    msg = "brick_cells incompatible with the cell grid";
    return ESP_ERR_INVALID_ARG;
  }
  if (n_c == 0) { msg = "no brick/tile shape fits in shared memory"; return ESP_ERR_UNSUPPORTED; }
  return ESP_OK;
}

// 2^32 / L as m 2^e with m a 64-bit integer (top bit set), rounded down: L =
// Lm 2^LE with Lm the 53-bit significand, so 2^32 / L = (2^k / Lm) 2^(32 - LE
// - k); the quotient is an exact 128-bit integer division (the same on every
// host).
static void fixed_scale(double L, unsigned long long& m, int& e) {
  int le = 0;
  const double f = std::frexp(L, &le);                   // L = f 2^le, f in [0.5, 1)
  const unsigned long long lm = (unsigned long long)std::ldexp(f, 53);   // exact
  int k = 116;
  if (lm == (1ull << 52)) k = 115;                      // 2^116 / 2^52 would need 65 bits
  const unsigned __int128 q = ((unsigned __int128)1 << k) / lm;
  m = (unsigned long long)q;
  e = 32 - (le - 53) - k;
}

esp_status make_host_plan(double L, long long N, double tol, const esp_plan_opts& o, HostPlan& hp,
                          std::string& msg) {
  if (!(L > 0.0) || !std::isfinite(L)) { msg = "box edge must be positive and finite"; return ESP_ERR_INVALID_ARG; }
  if (N < 0 || N >= (1LL << 31)) { msg = "N must be in [0, 2^31)"; return ESP_ERR_INVALID_ARG; }
  if (!(tol > 1e-15 && tol < 0.1)) { msg = "tolerance must be in (1e-15, 0.1)"; return ESP_ERR_INVALID_ARG; }
  const int prec = o.precision;
  const int kernel = o.kernel;
  if (prec != ESP_FP32 && prec != ESP_FP64) { msg = "precision must be ESP_FP32 or ESP_FP64"; return ESP_ERR_INVALID_ARG; }
  if (kernel != ESP_KERNEL_PSWF && kernel != ESP_KERNEL_GAUSS) { msg = "unknown kernel"; return ESP_ERR_INVALID_ARG; }
  const int pmax = prec == ESP_FP32 ? 12 : 16;

  if (o.window != ESP_WINDOW_PSWF && o.window != ESP_WINDOW_BSPLINE) { msg = "unknown SI window"; return ESP_ERR_INVALID_ARG; }
  if (o.diff != ESP_DIFF_AD && o.diff != ESP_DIFF_IK) { msg = "diff must be ESP_DIFF_AD or ESP_DIFF_IK"; return ESP_ERR_INVALID_ARG; }
  if (o.virial != 0 && o.virial != 1) { msg = "virial must be 0 or 1"; return ESP_ERR_INVALID_ARG; }
  if (o.virial && (prec == ESP_FP32 ? (o.near_variant != 0 && o.near_variant != 4)
                                    : (o.near_variant != 0 && o.near_variant != 1))) {
    msg = "the virial needs the default local-part kernel";
    return ESP_ERR_UNSUPPORTED;
  }
  const bool bspline = o.window == ESP_WINDOW_BSPLINE;
  const double c = o.c > 0 ? o.c : cached_c(tol);
  // the B-spline comparator defaults to order 5, the MD packages' default
  const int P = o.P > 0 ? o.P : (bspline ? 5 : espm::stencil_width(tol));
  if (P < espk::kMinP || P > pmax) {
    msg = "stencil width P=" + std::to_string(P) + " outside the compiled range [4, " + std::to_string(pmax) + "]";
    return ESP_ERR_UNSUPPORTED;
  }
  const double alpha = kernel == ESP_KERNEL_GAUSS ? (o.alpha > 0 ? o.alpha : std::log(1.0 / tol)) : 0.0;
  espm::Split split = kernel == ESP_KERNEL_PSWF ? cached_pswf_split(c) : espm::make_gauss_split(alpha);

  double r_c = o.r_c;
  if (!(r_c > 0)) {
    double best = 1e300;
    r_c = 0.45 * L;
    for (int i = 0; i < 60; ++i) {
      const double r = L * (0.02 + (0.48 - 0.02) * i / 59.0);
      const double t = model_cost(L, std::max<long long>(N, 1), P, c, r, kernel, tol);
      if (t < best) { best = t; r_c = r; }
    }
  }
  if (!(r_c < 0.5 * L)) { msg = "cutoff r_c must be smaller than L/2"; return ESP_ERR_CUTOFF_TOO_LARGE; }

  // grid size and SI-kernel shape
  RadialChihat chi(split, L, r_c);
  std::vector<double> ratios;
  if (o.c1 > 0) ratios.push_back(o.c1 / c);
  else for (int i = 0; i < 7; ++i) ratios.push_back(1.10 + 0.05 * i);
  int n_f;
  if (o.n_f > 0) {
    if (o.n_f % 2 || o.n_f < 4) { msg = "n_f must be even and >= 4"; return ESP_ERR_INVALID_ARG; }
    n_f = o.n_f;
  } else {
    const double nmin = kernel == ESP_KERNEL_PSWF ? c * L / (kPi * r_c)
                                                  : 2.0 * std::ceil(std::log(1.0 / tol) * L / (kPi * r_c));
    n_f = espm::round_grid(std::max(4.0, nmin));
  }
  if (n_f > 1024) { msg = "grid too large (n_f > 1024): raise r_c or the tolerance"; return ESP_ERR_UNSUPPORTED; }
  double best_c1 = ratios[0] * c, best_alias = 1e300;
  espm::Window bwin;
  if (bspline) {
    // B-spline window (the "Default" comparator): no shape to choose; unless
    // n_f is given, the grid is the one Table 2 says the default PME needs
    // for the same error, R_default^(1/3) times ESP's c L / (pi r_c) (and at
    // least the Gaussian truncation minimum); the aliasing estimate at that
    // grid is reported
    bwin = espm::make_bspline_window(P);
    best_c1 = 0.0;
    if (o.n_f == 0) {
      const double c_esp = cached_c(tol);
      const double nmin = std::max(2.0 * std::ceil(std::log(1.0 / tol) * L / (kPi * r_c)),
                                   espm::default_grid_ratio(tol) * c_esp * L / (kPi * r_c));
      n_f = espm::round_grid(std::max(4.0, nmin));
      if (n_f > 1024) { msg = "grid too large (n_f > 1024): raise r_c or the tolerance"; return ESP_ERR_UNSUPPORTED; }
    }
    best_alias = alias_from_rows(alias_rows(chi, n_f), bwin, n_f);
  } else {
    std::vector<espm::Window> windows;
    for (double r : ratios) windows.push_back(cached_window(r * c, P));
    for (int step = 0; step < 8; ++step) {
      const std::vector<double> rows = alias_rows(chi, n_f);
      best_alias = 1e300;
      for (size_t i = 0; i < ratios.size(); ++i) {
        const double a = alias_from_rows(rows, windows[i], n_f);
        if (a < best_alias) { best_alias = a; best_c1 = ratios[i] * c; }
      }
      if (o.n_f > 0 || best_alias <= 0.5 * tol || n_f >= 1024) break;
      n_f = espm::round_grid(n_f + 1);
    }
  }
  const espm::Window win = bspline ? bwin : cached_window(best_c1, P);

  // cell list and bricks: cell edge w >= r_c / reach. For the one-thread-per-
  // atom local part a reach of 3 (smaller cells) reads fewer non-neighbours;
  // the cluster form lists whole columns and runs faster with reach 2 (fewer
  // ranges per cluster). Reach 3 needs a few cells per axis to pay off.
  const bool cluster_form = prec == ESP_FP32 && (o.near_variant >= 3 || o.near_variant == 0);
  int reach = o.cell_reach > 0 ? o.cell_reach : (cluster_form ? 2 : 3);
  if (reach < 1 || reach > 4) { msg = "cell_reach must be 1 ... 4"; return ESP_ERR_INVALID_ARG; }
  if (o.cell_reach <= 0 && std::floor(3.0 * L / r_c) < 9) reach = 2;
  // the local part keeps per-axis cell tables in shared memory (512 entries)
  if (o.cell_reach <= 0) while (reach > 1 && std::floor(reach * L / r_c) > 512) --reach;
  if (std::floor(reach * L / r_c) > 512) {
    msg = "more than 512 cell-list cells per axis: raise r_c or lower cell_reach";
    return ESP_ERR_UNSUPPORTED;
  }
  const int nc_max = std::max(1, (int)std::floor(reach * L / r_c * (1.0 - 1e-12)));
  const double h = L / n_f;
  int n_c = 0, bc = 0, T = 0;
  {
    const esp_status bs = choose_bricks(n_f, nc_max, L, P, o, n_c, bc, T, msg);
    if (bs != ESP_OK) return bs;
  }

  // descriptor
  espk::SysDesc& d = hp.desc;
  d = espk::SysDesc{};
  d.n_f = n_f; d.n_c = n_c; d.bc = bc; d.nb = n_c / bc; d.T = T;
  espk::tile_pitches(T, P, d.tpy, d.tpz);
  d.reach = reach;
  d.n_atoms = (int)N;
  d.gsize = 3 * (n_f / 2) * (n_f / 2) + 1;
  d.L = L; d.inv_L = 1.0 / L; d.h = h; d.inv_h = n_f / L;
  d.vol = L * L * L;
  d.r_c = r_c; d.rc2 = r_c * r_c; d.inv_rc = 1.0 / r_c;
  d.inv_rc2 = d.inv_rc * d.inv_rc; d.inv_rc3 = d.inv_rc2 * d.inv_rc;
  d.w = L / n_c;
  d.fix_scale = L / 4294967296.0;
  d.to_fixed = 4294967296.0 / L;
  fixed_scale(L, d.fix_m, d.fix_e);
  d.w32 = d.w / 4294967296.0;
  d.wf = (float)d.w;
  d.w32f = d.wf * 2.3283064365386962890625e-10f;
  d.r_cf = (float)r_c;
  d.rc2f = (float)d.rc2;
  d.inv_rcf = (float)d.inv_rc;
  d.inv_rc2x2f = (float)(2.0 * d.inv_rc2);
  d.inv_rc3f = (float)d.inv_rc3;
  d.inv_bcf = (float)(1.0 / bc);
  hp.self_unit = split.chi0() / (4.0 * kPi * r_c);
  hp.m2 = split.second_moment();
  d.self_coef = hp.self_unit;
  d.bg_shift = 0.0;
  d.prefactor = o.prefactor > 0 ? o.prefactor : 1.0;
  d.self_coef_f = (float)d.self_coef;
  d.bg_shift_f = 0.0f;
  d.prefactor_f = (float)d.prefactor;

  // polynomial tables
  const SiTables& sit = si_tables(win, P);
  hp.si32 = sit.si32;
  hp.si64 = sit.si64;
  const double si_err = prec == ESP_FP32 ? sit.err32 : sit.err64;
  const NearTables& nt = near_tables(split, tol);
  hp.nc32 = nt.nc32;
  hp.nc64 = nt.nc64;
  hp.near_nc = prec == ESP_FP32 ? nt.terms32 : espk::Deg<double>::nr;
  const double near_err = prec == ESP_FP32 ? nt.err32 : nt.err64;

  // influence tables (Eq. pk, Phi in grid units); the virial table only for
  // plans that form the virial (zeros otherwise: the scale kernel reads it
  // only then)
  hp.G.assign(d.gsize, 0.0);
  hp.H.assign(d.gsize, 0.0);
  chi(d.gsize - 1);
  for (int m = 1; m < d.gsize; ++m) {
    const double xi = 2.0 * kPi * std::sqrt((double)m) / L;
    const double ch = chi(m);
    hp.G[m] = ch / (xi * xi) / (L * L * L);
    // virial: (r_c xi chihat'(r_c xi) - 2 chihat(r_c xi)) / (xi^2 L^3)
    if (o.virial) hp.H[m] = (r_c * xi * split.dchihat(r_c * xi) - 2.0 * ch) / (xi * xi) / (L * L * L);
  }
  hp.W.assign(n_f / 2 + 1, 0.0);
  for (int k = 0; k <= n_f / 2; ++k) {
    const double ph = win.Phi(2.0 * kPi * k / n_f);
    hp.W[k] = 1.0 / (ph * ph);
  }

  hp.tol = tol;
  if (o.near_variant < 0 || o.near_variant > 4) { msg = "near_variant must be 0 ... 4"; return ESP_ERR_INVALID_ARG; }
  hp.near_queued = o.near_variant == 2;
  hp.near_clusters = prec == ESP_FP32 && (o.near_variant >= 3 || o.near_variant == 0);
  hp.near_half = hp.near_clusters && o.near_variant != 3;
  hp.n_keys = (long long)n_c * n_c * n_c * espk::kSub;
  hp.grid_elems = (long long)n_f * n_f * n_f;
  hp.spec_elems = (long long)n_f * n_f * (n_f / 2 + 1);
  hp.n_bricks = d.nb * d.nb * d.nb;

  esp_plan_params& info = hp.info;
  info = esp_plan_params{};
  info.L = L; info.r_c = r_c; info.h = h; info.c = c; info.c1 = best_c1; info.alpha = alpha;
  info.prefactor = d.prefactor;
  info.alias_estimate = best_alias;
  info.si_fit_error = si_err;
  info.near_fit_error = near_err;
  info.N = N; info.P = P; info.n_f = n_f; info.kernel = kernel; info.precision = prec;
  info.n_cells = n_c; info.brick_cells = bc; info.tile = T;
  info.cell_reach = reach; info.near_terms = hp.near_nc;
  info.si_degree = (prec == ESP_FP32 ? espk::Deg<float>::si : espk::Deg<double>::si) - 1;
  info.window = o.window;
  info.diff = o.diff;
  info.virial = o.virial;
  info.near_degree = (prec == ESP_FP32 ? espk::Deg<float>::nr : espk::Deg<double>::nr) - 1;
  return ESP_OK;
}

// ------------------------------------------------------------ triclinic cell
// Influence over the half spectrum of a triclinic cell (Eq. pk with
// |xi(k)| = 2 pi |H^-T k| and Phi in grid units per fractional axis):
// G[idx] = chihat(r_c |xi|) / (|xi|^2 V) at the index order of the scale
// kernel ([kz][ky][kx], kx in [0, n_f/2]), with the mode set
// k_a in {-n_f/2, ..., n_f/2 - 1}. On a sheared lattice |xi(k)| is not even
// in a single component, so where a component is -n_f/2 the mode and the
// representative of -k carry different values; the real part of the inverse
// transform averages them, and G holds that average (the scaled spectrum is
// then exactly Hermitian, as the C2R transform assumes). chihat of the PSWF
// split comes from a cubic Hermite table in kappa (step 0.01; the fourth
// derivative of chihat is bounded by int_0^1 x^4 chi <= 1, so the table
// error is below 3e-11); the Gaussian split has its closed form.
static void triclinic_influence(const espm::Split& split, int n_f, const double Hi[6], double V, double r_c,
                                std::vector<double>& G) {
  const int nh = n_f / 2 + 1, half = n_f / 2;
  const double twopi = 2.0 * kPi;
  auto xi2_of = [&](int kx, int ky, int kz) {
    // H^-T k with H^-1 = [[i00, i01, i02], [0, i11, i12], [0, 0, i22]]
    const double vx = Hi[0] * kx;
    const double vy = Hi[1] * kx + Hi[3] * ky;
    const double vz = Hi[2] * kx + Hi[4] * ky + Hi[5] * kz;
    return twopi * twopi * (vx * vx + vy * vy + vz * vz);
  };
  // signed component of an index, and of the representative of its negative
  auto comp = [&](int i) { return i < half ? i : i - n_f; };
  auto neg = [&](int k) { return k == -half ? -half : -k; };
  double xi2_max = 0.0;
  for (int kz = -half; kz < half; ++kz)
    for (int ky = -half; ky < half; ++ky)
      for (int kx = -half; kx < half; ++kx) xi2_max = std::max(xi2_max, xi2_of(kx, ky, kz));
  const double step = 0.01;
  const bool table = split.kind != 1;
  std::vector<double> f, df;
  if (table) {
    const int nt = (int)std::ceil(r_c * std::sqrt(xi2_max) / step) + 2;
    f.resize(nt);
    df.resize(nt);
    for (int i = 0; i < nt; ++i) {
      f[i] = split.chihat(i * step);
      df[i] = split.dchihat(i * step);
    }
  }
  auto chihat = [&](double kappa) {
    if (!table) return split.chihat(kappa);
    const double x = kappa / step;
    const int i = std::min((int)x, (int)f.size() - 2);
    const double t = x - i, t2 = t * t, t3 = t2 * t;
    return (2 * t3 - 3 * t2 + 1) * f[i] + (t3 - 2 * t2 + t) * step * df[i] + (-2 * t3 + 3 * t2) * f[i + 1] +
           (t3 - t2) * step * df[i + 1];
  };
  auto p_of = [&](int kx, int ky, int kz) {
    const double xi2 = xi2_of(kx, ky, kz);
    return xi2 > 0.0 ? chihat(r_c * std::sqrt(xi2)) / xi2 / V : 0.0;
  };
  G.assign((size_t)n_f * n_f * nh, 0.0);
  size_t idx = 0;
  for (int kzi = 0; kzi < n_f; ++kzi)
    for (int kyi = 0; kyi < n_f; ++kyi)
      for (int kxi = 0; kxi < nh; ++kxi, ++idx) {
        const int kx = comp(kxi), ky = comp(kyi), kz = comp(kzi);
        const double p = p_of(kx, ky, kz);
        G[idx] = (kx == -half || ky == -half || kz == -half) ? 0.5 * (p + p_of(neg(kx), neg(ky), neg(kz))) : p;
      }
}

esp_status make_host_plan_cell(const double cell[9], long long N, double tol, const esp_plan_opts& o,
                               HostPlan& hp, std::string& msg) {
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) { msg = "cell vectors must be finite"; return ESP_ERR_INVALID_ARG; }
  const double ax = cell[0], bx = cell[3], by = cell[4], cx = cell[6], cy = cell[7], cz = cell[8];
  if (cell[1] != 0.0 || cell[2] != 0.0 || cell[5] != 0.0 || !(ax > 0) || !(by > 0) || !(cz > 0)) {
    msg = "cell vectors must be a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz) with ax, by, cz > 0";
    return ESP_ERR_INVALID_ARG;
  }
  if (o.precision != ESP_FP32) { msg = "triclinic cells need ESP_FP32"; return ESP_ERR_UNSUPPORTED; }
  if (o.diff != ESP_DIFF_AD) { msg = "triclinic cells use AD forces"; return ESP_ERR_UNSUPPORTED; }
  if (o.virial) { msg = "no virial on a triclinic cell"; return ESP_ERR_UNSUPPORTED; }
  if (o.near_variant != 0 && o.near_variant != 4) {
    msg = "triclinic cells need the default local-part kernel";
    return ESP_ERR_UNSUPPORTED;
  }
  // heights (distances between opposite faces) and the longest cell vector
  const double V = ax * by * cz;
  const double la = ax, lb = std::sqrt(bx * bx + by * by), lc = std::sqrt(cx * cx + cy * cy + cz * cz);
  const double bxc = std::sqrt((by * cz) * (by * cz) + (bx * cz) * (bx * cz) + (bx * cy - by * cx) * (bx * cy - by * cx));
  const double cxa = ax * std::sqrt(cz * cz + cy * cy);
  const double hx = V / bxc, hy = V / cxa, hz = cz;
  const double h_min = std::min(hx, std::min(hy, hz));
  const double L_eff = std::max(la, std::max(lb, lc));
  // parameters from the cubic rules on the longest cell vector (the grid
  // resolves every fractional axis at least as finely as a cube of that edge)
  esp_plan_opts o2 = o;
  if (!(o2.r_c > 0)) {
    HostPlan probe;
    const esp_status st = make_host_plan(L_eff, N, tol, o2, probe, msg);
    if (st != ESP_OK) return st;
    o2.r_c = std::min(probe.info.r_c, 0.45 * h_min);
  }
  const double r_c = o2.r_c;
  if (!(r_c < 0.5 * h_min)) {
    msg = "cutoff r_c must be smaller than half the smallest cell height";
    return ESP_ERR_CUTOFF_TOO_LARGE;
  }
  esp_status st = make_host_plan(L_eff, N, tol, o2, hp, msg);
  if (st != ESP_OK) return st;
  const int n_f = hp.info.n_f, P = hp.info.P;
  if (n_f > 384) {
    msg = "grid too large for a triclinic influence array (n_f > 384): raise r_c or the tolerance";
    return ESP_ERR_UNSUPPORTED;
  }
  // cells of fractional coordinates: a pair within r_c is at most r_c n_c / h_a
  // cells apart along axis a, so n_c <= reach h_min / r_c keeps it within reach
  const int reach = hp.desc.reach;
  const int nc_max = std::max(1, (int)std::floor(reach * h_min / r_c * (1.0 - 1e-12)));
  int n_c = 0, bc = 0, T = 0;
  st = choose_bricks(n_f, nc_max, L_eff, P, o2, n_c, bc, T, msg);
  if (st != ESP_OK) return st;

  espk::SysDesc& d = hp.desc;
  d.n_c = n_c; d.bc = bc; d.nb = n_c / bc; d.T = T;
  espk::tile_pitches(T, P, d.tpy, d.tpz);
  d.w = h_min / n_c;                 // smallest cell height (margins of the local part)
  d.wf = (float)d.w;
  d.w32 = d.w / 4294967296.0;
  d.w32f = d.wf * 2.3283064365386962890625e-10f;
  d.inv_bcf = (float)(1.0 / bc);
  d.vol = V;
  d.tri = 1;
  const double Hi[6] = {1.0 / ax, -bx / (ax * by), (bx * cy - by * cx) / (ax * by * cz),
                        1.0 / by, -cy / (by * cz), 1.0 / cz};
  for (int k = 0; k < 6; ++k) d.tfix[k] = 4294967296.0 * Hi[k];
  const double e[6] = {ax, bx, by, cx, cy, cz};
  for (int k = 0; k < 6; ++k) d.tcell[k] = e[k] / n_c;
  // n_f H^-T, lower triangle row by row: (xx), (yx, yy), (zx, zy, zz)
  const double g[6] = {Hi[0], Hi[1], Hi[3], Hi[2], Hi[4], Hi[5]};
  for (int k = 0; k < 6; ++k) d.tgrad[k] = (float)(n_f * g[k]);
  d.tcol[0] = (float)(ax / n_c);
  d.tcol[1] = (float)(bx / n_c);
  d.tcol[2] = (float)(by / n_c);
  d.tbrick[0] = (float)(bc * cx / n_c);
  d.tbrick[1] = (float)(bc * cy / n_c);
  d.tbrick[2] = (float)(bc * cz / n_c);

  // influence over the whole half spectrum (no virial table)
  const espm::Split split = o2.kernel == ESP_KERNEL_PSWF ? cached_pswf_split(hp.info.c)
                                                         : espm::make_gauss_split(hp.info.alpha);
  triclinic_influence(split, n_f, Hi, V, r_c, hp.G);
  d.gsize = (int)hp.G.size();
  hp.H.clear();
  hp.n_keys = (long long)n_c * n_c * n_c * espk::kSub;
  hp.n_bricks = d.nb * d.nb * d.nb;

  esp_plan_params& info = hp.info;
  info.L = L_eff;
  info.n_cells = n_c;
  info.brick_cells = bc;
  info.tile = T;
  info.triclinic = 1;
  return ESP_OK;
}

void charge_constants(const HostPlan& hp, double Q, double Q2, double* e_self, double* e_bg,
                      double* bg_shift) {
  const double V = hp.desc.vol, r_c = hp.desc.r_c;
  const double shift = -(Q / V) * 0.5 * r_c * r_c * hp.m2;
  *bg_shift = shift;
  *e_self = -0.5 * Q2 * hp.self_unit;
  *e_bg = 0.5 * Q * shift;
}

}  // namespace espe
