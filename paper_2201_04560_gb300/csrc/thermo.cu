// Host-side tools of the mesh-refinement procedure (arXiv 2201.04560, Sec. 3): the
// sigma that keeps the planar coexistence on the Maxwell densities (Eq.
// integral_coexistence_curve, secant from -16 G sigma_0 = 2), the planar surface tension
// (Eq. surface_tension) and the kappa of a refined mesh (Eq. gamma-meshes-relation), and
// the field scaling of Table 1 (a ~ dx^2, T ~ dx^2, g ~ dx^3). All FP64, no GPU.
//
// Quadrature: composite Gauss-Legendre (8 nodes per panel) for the coexistence integral;
// a fine cumulative trapezoid in rho for the planar profile integral.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/ppl.h"

namespace {

struct Pr {
  double a, b, R, omega, G, T, Tc, k, aa;  // aa = a alpha(T)
  double p(double r) const { return r * R * T / (1.0 - b * r) - aa * r * r / (1.0 + 2.0 * b * r - b * b * r * r); }
  double dp(double r) const {
    const double d = 1.0 + 2.0 * b * r - b * b * r * r;
    return R * T / ((1.0 - b * r) * (1.0 - b * r)) - aa * (2.0 * r * d - r * r * (2.0 * b - 2.0 * b * b * r)) / (d * d);
  }
  double psi2(double r) const { return 2.0 * (p(r) - r / 3.0) / G; }  // Eq. (psi) squared
  double psi(double r) const { return std::sqrt(std::fmax(psi2(r), 0.0)); }
  // d psi / d rho = (dp/drho - 1/3) / (G psi)
  double dpsi(double r) const { return (dp(r) - 1.0 / 3.0) / (G * psi(r)); }
};

bool make_pr(double a, double b, double R, double omega, double G, double T, Pr *e) {
  if (!(a > 0) || !(b > 0) || !(R > 0) || !(G < 0) || !(T > 0)) return false;
  e->a = a;
  e->b = b;
  e->R = R;
  e->omega = omega;
  e->G = G;
  e->T = T;
  e->Tc = ppl_tc(a, b, R);
  if (!(T < e->Tc)) return false;
  e->k = 0.37464 + 1.54226 * omega - 0.2699 * omega * omega;
  const double ar = 1.0 + e->k * (1.0 - std::sqrt(T / e->Tc));
  e->aa = a * ar * ar;
  return true;
}

// 8-point Gauss-Legendre nodes/weights on [-1, 1]
const double GLX[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                       0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
const double GLW[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                       0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

template <typename F>
double gauss(F f, double lo, double hi, int panels) {
  double s = 0.0;
  const double h = (hi - lo) / panels;
  for (int p = 0; p < panels; ++p) {
    const double c = lo + (p + 0.5) * h;
    for (int i = 0; i < 8; ++i) s += GLW[i] * f(c + 0.5 * h * GLX[i]);
  }
  return 0.5 * h * s;
}

// Eq. (integral_coexistence_curve) at given (rho_v, rho_l, p0): int (p0 - p) psi' / psi^(1 - 16 G sigma)
double coexistence_integral(const Pr &e, double sigma, double rv, double rl, double p0) {
  const double ex = 1.0 - 16.0 * e.G * sigma;
  return gauss([&](double r) { return (p0 - e.p(r)) * e.dpsi(r) / std::pow(e.psi(r), ex); }, rv, rl, 2000);
}

template <typename F>
double bisect(F f, double lo, double hi) {
  double flo = f(lo);
  for (int it = 0; it < 300; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double fm = f(mid);
    if ((fm > 0) == (flo > 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
    if (hi - lo <= 1e-16 * std::fabs(hi)) break;
  }
  return 0.5 * (lo + hi);
}

// spinodal densities (local max / min of the isotherm)
bool spinodal(const Pr &e, double *rmax, double *rmin) {
  const double top = 0.999999 / e.b;
  const int n = 20000;
  double ra = -1, rb = -1;
  for (int i = 1; i < n; ++i) {
    const double r0 = top * (i - 1) / n + 1e-12, r1 = top * i / n;
    if (ra < 0 && e.dp(r0) > 0 && e.dp(r1) <= 0) ra = r1;
    if (ra > 0 && e.dp(r0) < 0 && e.dp(r1) >= 0) {
      rb = r1;
      break;
    }
  }
  if (ra < 0 || rb < 0) return false;
  *rmax = bisect([&](double r) { return e.dp(r); }, ra - top / n, ra);
  *rmin = bisect([&](double r) { return e.dp(r); }, rb - top / n, rb);
  return true;
}

// coexistence selected by the weighted equal-area condition int (p0 - p) w(rho) d rho = 0
template <typename Wt>
bool equal_area(const Pr &e, Wt w, double *rv, double *rl, double *p0) {
  double smax, smin;
  if (!spinodal(e, &smax, &smin)) return false;
  const double top = 0.999999 / e.b;
  const double phi = e.p(smax), plo = std::fmax(e.p(smin), 1e-300);
  double v = 0, l = 0;
  auto g = [&](double ps) {
    v = bisect([&](double r) { return e.p(r) - ps; }, 1e-300, smax);
    l = bisect([&](double r) { return e.p(r) - ps; }, smin, top);
    return gauss([&](double r) { return (ps - e.p(r)) * w(r); }, v, l, 2000);
  };
  const double eps = 1e-12 * (phi - plo);
  const double ps = bisect(g, plo + eps, phi - eps);
  g(ps);
  *rv = v;
  *rl = l;
  *p0 = ps;
  return true;
}

}  // namespace

extern "C" {

int ppl_sigma_for(double a, double b, double R, double omega, double G, double T, double *sigma) {
  Pr e;
  if (!sigma || !make_pr(a, b, R, omega, G, T, &e)) return PPL_E_INVAL;
  double rv, rl, ps;
  if (ppl_maxwell(a, b, R, omega, T, &rv, &rl, &ps) != PPL_OK) return PPL_E_INVAL;
  // secant on sigma, started at -16 G sigma_0 = 2 (second iterate 1% away)
  double s0 = -2.0 / (16.0 * G), s1 = 0.99 * s0;
  double f0 = coexistence_integral(e, s0, rv, rl, ps), f1 = coexistence_integral(e, s1, rv, rl, ps);
  for (int it = 0; it < 100; ++it) {
    if (f1 == f0) break;
    const double s2 = s1 - f1 * (s1 - s0) / (f1 - f0);
    s0 = s1;
    f0 = f1;
    s1 = s2;
    f1 = coexistence_integral(e, s1, rv, rl, ps);
    if (std::fabs(s1 - s0) < 1e-13 * std::fmax(1.0, std::fabs(s1))) {
      *sigma = s1;
      return PPL_OK;
    }
  }
  return PPL_E_INVAL;
}

int ppl_gamma_planar(double a, double b, double R, double omega, double G, double T, double sigma, double kappa,
                     double *gamma) {
  Pr e;
  if (!gamma || !make_pr(a, b, R, omega, G, T, &e)) return PPL_E_INVAL;
  // mechanical coexistence at this sigma (weight psi' / psi^(1 - 16 G sigma))
  const double ex = 1.0 - 16.0 * G * sigma;
  double rv, rl, p0;
  if (!equal_area(e, [&](double r) { return e.dpsi(r) / std::pow(e.psi(r), ex); }, &rv, &rl, &p0))
    return PPL_E_INVAL;
  // planar normal stress p + 2 sigma G^2 psi'^2 + (G/4) psi psi'' = p0 (c = 1); with Y = (d psi/dx)^2
  // as a function of psi: d(Y psi^e)/d psi = (8 / (G psi)) (p0 - p) psi^e, e = 16 G sigma,
  // integrated in rho by a cumulative trapezoid; gamma = -(G/6)(1 - kappa) int sqrt(Y) d psi
  const double e2 = 16.0 * G * sigma;
  const int n = 400000;
  const double h = (rl - rv) / n;
  std::vector<double> src(n + 1), dps(n + 1), psv(n + 1), fwd(n + 1), bwd(n + 1);
  for (int i = 0; i <= n; ++i) {
    const double r = rv + i * h;
    psv[i] = e.psi(r);
    dps[i] = e.dpsi(r);
    src[i] = (8.0 / (G * psv[i])) * (p0 - e.p(r)) * std::pow(psv[i], e2) * dps[i];  // d/d rho of (Y psi^e)
  }
  // Y psi^e vanishes in both bulks: accumulate from the nearer end to avoid cancellation
  fwd[0] = 0.0;
  for (int i = 1; i <= n; ++i) fwd[i] = fwd[i - 1] + 0.5 * h * (src[i] + src[i - 1]);
  bwd[n] = 0.0;
  for (int i = n - 1; i >= 0; --i) bwd[i] = bwd[i + 1] - 0.5 * h * (src[i] + src[i + 1]);
  double gam = 0.0, prev = 0.0;
  for (int i = 0; i <= n; ++i) {
    const double Ye = i <= n / 2 ? fwd[i] : bwd[i];
    const double sq = std::sqrt(std::fmax(Ye, 0.0) * std::pow(psv[i], -e2)) * dps[i];
    if (i > 0) gam += 0.5 * h * (sq + prev);
    prev = sq;
  }
  *gamma = -(G / 6.0) * (1.0 - kappa) * gam;
  return PPL_OK;
}

int ppl_kappa_for(double a_base, int32_t n_base, int32_t n, double b, double R, double omega, double G,
                  double T_ratio, double kappa_base, double *kappa) {
  if (!kappa || n_base <= 0 || n <= 0 || !(T_ratio > 0 && T_ratio < 1)) return PPL_E_INVAL;
  const double a1 = ppl_refine_a(a_base, n_base, n);
  double s0, s1, g0, g1;
  const double T0 = T_ratio * ppl_tc(a_base, b, R), T1 = T_ratio * ppl_tc(a1, b, R);
  if (ppl_sigma_for(a_base, b, R, omega, G, T0, &s0) || ppl_sigma_for(a1, b, R, omega, G, T1, &s1) ||
      ppl_gamma_planar(a_base, b, R, omega, G, T0, s0, kappa_base, &g0) ||
      ppl_gamma_planar(a1, b, R, omega, G, T1, s1, 0.0, &g1))
    return PPL_E_INVAL;
  // Eq. (gamma-meshes-relation): gamma_1 = gamma_0 dx_1 / dx_0 with dx ~ 1/n; gamma ~ (1 - kappa)
  *kappa = 1.0 - g0 * ((double)n_base / n) / g1;
  return PPL_OK;
}

int ppl_refine(const ppl_config *base, int32_t n_base, int32_t n, double T_ratio, ppl_config *out) {
  if (!base || !out || n_base <= 0 || n <= 0 || !(T_ratio > 0 && T_ratio < 1)) return PPL_E_INVAL;
  for (int s = 0; s < 4; ++s)
    if (base->rho_w[s] || base->T_w[s] || base->T_dirichlet[s]) return PPL_E_INVAL;  // per-node arrays: caller
  const double r = (double)n / n_base;  // refinement ratio dx_0 / dx
  ppl_config c = *base;
  // Table 1: lengths ~ 1/dx, a ~ dx^2 (Eq. a-deltax), T and p ~ dx^2, g ~ dx^3; rho, lambda, c_v, eta O(1)
  c.nx = (int32_t)std::lround(base->nx * r);
  c.ny = (int32_t)std::lround(base->ny * r);
  c.a = ppl_refine_a(base->a, n_base, n);
  const double tsc = ppl_tc(c.a, c.b, c.R) / ppl_tc(base->a, base->b, base->R);
  for (int s = 0; s < 4; ++s) c.T_side[s] = base->T_side[s] * tsc;
  c.T_ref = base->T_ref * tsc;
  c.iso_steps = (int64_t)std::llround((double)base->iso_steps * r * r);  // dt ~ dx^2
  c.gx = base->gx / (r * r * r);
  c.gy = base->gy / (r * r * r);
  const double T = T_ratio * ppl_tc(c.a, c.b, c.R);
  if (ppl_sigma_for(c.a, c.b, c.R, c.omega, c.G, T, &c.sigma)) return PPL_E_INVAL;
  if (ppl_kappa_for(base->a, n_base, n, c.b, c.R, c.omega, c.G, T_ratio, base->kappa, &c.kappa)) return PPL_E_INVAL;
  *out = c;
  return PPL_OK;
}


int ppl_pressure(double a, double b, double R, double omega, double T, double rho, double *p, double *dp_drho) {
  Pr e;
  if (!(a > 0) || !(b > 0) || !(R > 0) || !(T > 0) || !(rho >= 0) || !(b * rho < 1.0)) return PPL_E_INVAL;
  e.a = a;
  e.b = b;
  e.R = R;
  e.omega = omega;
  e.G = -1.0;
  e.T = T;
  e.Tc = ppl_tc(a, b, R);
  e.k = 0.37464 + 1.54226 * omega - 0.2699 * omega * omega;
  const double ar = 1.0 + e.k * (1.0 - std::sqrt(T / e.Tc));
  e.aa = a * ar * ar;
  if (p) *p = e.p(rho);
  if (dp_drho) *dp_drho = e.dp(rho);
  return PPL_OK;
}

}  // extern "C"
