// Host FP64 cosmology for the PM lensing library.
//
// Flat LCDM without radiation, H0 = 1: E(a) = sqrt(Om a^-3 + 1 - Om).
// Linear growth (first and second order) is integrated with classical RK4 on
// a uniform grid in y = ln a, from a = 1e-5 (matter domination, growing modes
// D1 = a, D2 = -3/7 a^2) to a = 1, together with the comoving distance
// (Appendix A: chi = (c/H0) int dz / E).  In y the growth equations read
//   d2D/dy2 = -(2 + dlnE/dlna) dD/dy + (3/2) Om / (a^3 E^2) D
//   d2D2/dy2 = -(2 + dlnE/dlna) dD2/dy + (3/2) Om / (a^3 E^2) (D2 - D1^2)
// FastPM time factors (Sec. 3, "enforcing correct linear displacement"):
//   g_p = a^3 E dD1/da = a^2 E dD1/dy,   g_f = a^2 E dg_p/da.
// The linear power is the Eisenstein & Hu (1998) transfer function with
// baryon oscillations (Appendix A), normalised to sigma_8 with a real-space
// top-hat of radius 8 Mpc/h.
#include <cmath>

#include "pm_internal.h"

namespace pmlens {

double Cosmo::E(double a) const { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

double Cosmo::dlnE_dlna(double a) const {
  const double e = E(a);
  return -1.5 * om / (a * a * a * e * e);
}

namespace {
struct Y5 { double v[5]; };

Y5 rhs(const Cosmo& c, double y, const Y5& s) {
  const double a = std::exp(y);
  const double e = c.E(a);
  const double damp = 2.0 + c.dlnE_dlna(a);
  const double src = 1.5 * c.om / (a * a * a * e * e);
  Y5 d;
  d.v[0] = s.v[1];
  d.v[1] = -damp * s.v[1] + src * s.v[0];
  d.v[2] = s.v[3];
  d.v[3] = -damp * s.v[3] + src * (s.v[2] - s.v[0] * s.v[0]);
  d.v[4] = kCoverH0 / (a * e);  // d(chi_tilde)/dy, chi = chi_tilde(1) - chi_tilde(a)
  return d;
}

Y5 axpy(const Y5& x, double h, const Y5& d) {
  Y5 r;
  for (int i = 0; i < 5; ++i) r.v[i] = x.v[i] + h * d.v[i];
  return r;
}

inline double hermite(double y0, double y1, double d0, double d1, double h, double t) {
  const double t2 = t * t, t3 = t2 * t;
  return (2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * h * d0 + (-2 * t3 + 3 * t2) * y1 +
         (t3 - t2) * h * d1;
}

double tophat(double x) {
  if (x < 1e-4) return 1.0 - x * x / 10.0;
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}
}  // namespace

void Cosmo::init(double omega_m, double sigma8, double hh, double n_s, double omega_b,
                 double t_cmb) {
  om = omega_m; s8 = sigma8; h = hh; ns = n_s; ob = omega_b; tcmb = t_cmb;
  const double amin = 1e-5;
  n = 60000;
  lna0 = std::log(amin);
  dlna = -lna0 / n;
  d1.assign(n + 1, 0); d1d.assign(n + 1, 0); d2.assign(n + 1, 0); d2d.assign(n + 1, 0);
  chi.assign(n + 1, 0);
  Y5 s = {{amin, amin, -3.0 / 7.0 * amin * amin, -6.0 / 7.0 * amin * amin, 0.0}};
  std::vector<double> ct(n + 1);
  for (int k = 0; k <= n; ++k) {
    d1[k] = s.v[0]; d1d[k] = s.v[1]; d2[k] = s.v[2]; d2d[k] = s.v[3]; ct[k] = s.v[4];
    if (k == n) break;
    const double y = lna0 + k * dlna, hs = dlna;
    const Y5 k1 = rhs(*this, y, s);
    const Y5 k2 = rhs(*this, y + 0.5 * hs, axpy(s, 0.5 * hs, k1));
    const Y5 k3 = rhs(*this, y + 0.5 * hs, axpy(s, 0.5 * hs, k2));
    const Y5 k4 = rhs(*this, y + hs, axpy(s, hs, k3));
    for (int i = 0; i < 5; ++i) s.v[i] += hs / 6.0 * (k1.v[i] + 2 * k2.v[i] + 2 * k3.v[i] + k4.v[i]);
  }
  const double norm = d1[n];
  for (int k = 0; k <= n; ++k) {
    d1[k] /= norm; d1d[k] /= norm;
    d2[k] /= norm * norm; d2d[k] /= norm * norm;
    chi[k] = ct[n] - ct[k];
  }
  // sigma_8 normalisation: Simpson in ln k of k^3 T^2 k^ns W^2 / (2 pi^2)
  // (smooth integrand: 2e4 intervals over 21 e-folds give ~1e-12 relative error)
  const int nk = 20000;
  const double l0 = std::log(1e-6), l1 = std::log(1e3), hk = (l1 - l0) / nk;
  double acc = 0.0;
  for (int i = 0; i <= nk; ++i) {
    const double k = std::exp(l0 + i * hk);
    const double t = transfer(k);
    const double w = tophat(8.0 * k);
    const double f = std::pow(k, 3.0 + ns) * t * t * w * w / (2.0 * M_PI * M_PI);
    const double c = (i == 0 || i == nk) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    acc += c * f;
  }
  acc *= hk / 3.0;
  pk_norm = s8 * s8 / acc;
}

void Cosmo::state(double a, double* D1o, double* dD1o, double* D2o, double* dD2o) const {
  const double y = std::log(a);
  double u = (y - lna0) / dlna;
  int k = (int)std::floor(u);
  if (k < 0) k = 0;
  if (k > n - 1) k = n - 1;
  const double t = u - k;
  const double a0 = std::exp(lna0 + k * dlna), a1 = std::exp(lna0 + (k + 1) * dlna);
  // second derivatives from the ODE at the nodes (for the Hermite of dD/dy)
  auto dd = [&](double aa, double D, double dD, double D1v, bool second) {
    const double e = E(aa);
    const double damp = 2.0 + dlnE_dlna(aa);
    const double src = 1.5 * om / (aa * aa * aa * e * e);
    return second ? -damp * dD + src * (D - D1v * D1v) : -damp * dD + src * D;
  };
  const double dd1_0 = dd(a0, d1[k], d1d[k], 0, false), dd1_1 = dd(a1, d1[k + 1], d1d[k + 1], 0, false);
  const double dd2_0 = dd(a0, d2[k], d2d[k], d1[k], true);
  const double dd2_1 = dd(a1, d2[k + 1], d2d[k + 1], d1[k + 1], true);
  if (D1o) *D1o = hermite(d1[k], d1[k + 1], d1d[k], d1d[k + 1], dlna, t);
  if (dD1o) *dD1o = hermite(d1d[k], d1d[k + 1], dd1_0, dd1_1, dlna, t);
  if (D2o) *D2o = hermite(d2[k], d2[k + 1], d2d[k], d2d[k + 1], dlna, t);
  if (dD2o) *dD2o = hermite(d2d[k], d2d[k + 1], dd2_0, dd2_1, dlna, t);
}

double Cosmo::D1(double a) const { double v; state(a, &v, nullptr, nullptr, nullptr); return v; }
double Cosmo::D2(double a) const { double v; state(a, nullptr, nullptr, &v, nullptr); return v; }
double Cosmo::gp(double a) const {
  double dv; state(a, nullptr, &dv, nullptr, nullptr);
  return a * a * E(a) * dv;
}
double Cosmo::gp2(double a) const {
  double dv; state(a, nullptr, nullptr, nullptr, &dv);
  return a * a * E(a) * dv;
}
double Cosmo::gf(double a) const {
  // a^2 E d(a^2 E dD/dy)/da = a^3 E^2 [(2 + dlnE/dlna) dD/dy + d2D/dy2]
  double D, dD;
  state(a, &D, &dD, nullptr, nullptr);
  const double e = E(a);
  const double damp = 2.0 + dlnE_dlna(a);
  const double d2 = -damp * dD + 1.5 * om / (a * a * a * e * e) * D;
  return a * a * a * e * e * (damp * dD + d2);
}

double Cosmo::chi_a(double a) const {
  const double y = std::log(a);
  double u = (y - lna0) / dlna;
  int k = (int)std::floor(u);
  if (k < 0) k = 0;
  if (k > n - 1) k = n - 1;
  const double t = u - k;
  const double a0 = std::exp(lna0 + k * dlna), a1 = std::exp(lna0 + (k + 1) * dlna);
  const double c0 = -kCoverH0 / (a0 * E(a0)), c1 = -kCoverH0 / (a1 * E(a1));
  return hermite(chi[k], chi[k + 1], c0, c1, dlna, t);
}

void Cosmo::a_of_chi_grid(double h, int n, double* out) const {
  // chi decreases along the ln a grid: walk it once, then refine each entry by
  // Newton steps on chi(a) - c with dchi/dlna = -(c/H0) / (a E)
  int k = this->n;  // grid index, chi[k] <= c <= chi[k-1]
  for (int q = 0; q < n; ++q) {
    const double c = q * h;
    if (c <= 0) { out[q] = 1.0; continue; }
    while (k > 0 && chi[k - 1] < c) --k;
    if (k == 0) { out[q] = std::exp(lna0); continue; }
    // linear start between the bracketing nodes, then Newton in y = ln a
    const double f = (c - chi[k]) / (chi[k - 1] - chi[k]);
    double y = lna0 + (k - f) * dlna;
    for (int it = 0; it < 4; ++it) {
      const double a = std::exp(y);
      const double g = chi_a(a) - c;
      y += g * a * E(a) / kCoverH0;
    }
    out[q] = std::exp(y);
  }
}

double Cosmo::a_of_chi(double c) const {
  double lo = 1e-5, hi = 1.0;  // chi decreasing in a
  if (c <= 0) return 1.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (chi_a(mid) > c) lo = mid; else hi = mid;
    if (hi - lo < 1e-15) break;
  }
  return 0.5 * (lo + hi);
}

double Cosmo::transfer(double k_hmpc) const {
  // Eisenstein & Hu (1998), ApJ 496, 605: fitting formulae in Mpc^-1.
  const double k = k_hmpc * h;
  const double w_m = om * h * h, w_b = ob * h * h;
  const double fb = ob / om, fc = 1.0 - fb;
  const double th = tcmb / 2.7;
  const double zeq = 2.50e4 * w_m * std::pow(th, -4.0);
  const double keq = 7.46e-2 * w_m * std::pow(th, -2.0);
  const double bd1 = 0.313 * std::pow(w_m, -0.419) * (1.0 + 0.607 * std::pow(w_m, 0.674));
  const double bd2 = 0.238 * std::pow(w_m, 0.223);
  const double zd = 1291.0 * std::pow(w_m, 0.251) / (1.0 + 0.659 * std::pow(w_m, 0.828)) *
                    (1.0 + bd1 * std::pow(w_b, bd2));
  const double Req = 31.5 * w_b * std::pow(th, -4.0) * 1e3 / zeq;
  const double Rd = 31.5 * w_b * std::pow(th, -4.0) * 1e3 / zd;
  const double s = 2.0 / (3.0 * keq) * std::sqrt(6.0 / Req) *
                   std::log((std::sqrt(1.0 + Rd) + std::sqrt(Rd + Req)) / (1.0 + std::sqrt(Req)));
  const double ksilk = 1.6 * std::pow(w_b, 0.52) * std::pow(w_m, 0.73) *
                       (1.0 + std::pow(10.4 * w_m, -0.95));
  if (k <= 0) return 1.0;
  const double q = k / (13.41 * keq);
  auto T0 = [&](double alpha, double beta) {
    const double L = std::log(M_E + 1.8 * beta * q);
    const double C = 14.2 / alpha + 386.0 / (1.0 + 69.9 * std::pow(q, 1.08));
    return L / (L + C * q * q);
  };
  const double a1 = std::pow(46.9 * w_m, 0.670) * (1.0 + std::pow(32.1 * w_m, -0.532));
  const double a2 = std::pow(12.0 * w_m, 0.424) * (1.0 + std::pow(45.0 * w_m, -0.582));
  const double alpha_c = std::pow(a1, -fb) * std::pow(a2, -fb * fb * fb);
  const double bc1 = 0.944 / (1.0 + std::pow(458.0 * w_m, -0.708));
  const double bc2 = std::pow(0.395 * w_m, -0.0266);
  const double beta_c = 1.0 / (1.0 + bc1 * (std::pow(fc, bc2) - 1.0));
  const double ks = k * s;
  const double f = 1.0 / (1.0 + std::pow(ks / 5.4, 4.0));
  const double Tc = f * T0(1.0, beta_c) + (1.0 - f) * T0(alpha_c, beta_c);
  const double y = (1.0 + zeq) / (1.0 + zd);
  const double sq = std::sqrt(1.0 + y);
  const double G = y * (-6.0 * sq + (2.0 + 3.0 * y) * std::log((sq + 1.0) / (sq - 1.0)));
  const double alpha_b = 2.07 * keq * s * std::pow(1.0 + Rd, -0.75) * G;
  const double beta_node = 8.41 * std::pow(w_m, 0.435);
  const double beta_b = 0.5 + fb + (3.0 - 2.0 * fb) * std::sqrt(std::pow(17.2 * w_m, 2.0) + 1.0);
  const double st = s / std::cbrt(1.0 + std::pow(beta_node / ks, 3.0));
  const double x = k * st;
  const double j0 = x > 1e-8 ? std::sin(x) / x : 1.0;
  const double Tb = (T0(1.0, 1.0) / (1.0 + (ks / 5.2) * (ks / 5.2)) +
                     alpha_b / (1.0 + std::pow(beta_b / ks, 3.0)) * std::exp(-std::pow(k / ksilk, 1.4))) *
                    j0;
  return fb * Tb + fc * Tc;
}

double Cosmo::pk(double k_hmpc) const {
  if (k_hmpc <= 0) return 0.0;
  const double t = transfer(k_hmpc);
  return pk_norm * std::pow(k_hmpc, ns) * t * t;
}

}  // namespace pmlens
