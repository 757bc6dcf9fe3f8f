"""Thermodynamic tools of the oracle (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY: this module is part of the CPU oracle. Only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it. The product path (the CUDA library and its binding) never does.

Each function restates one definition of arXiv 2201.04560 (Jaramillo,
Mapelli, Cabezas-Gomez, "Pseudopotential LBM for boiling heat transfer: a mesh
refinement procedure") in plain, slow, readable form:

* Peng-Robinson EOS, Sec. 2.1 Eq. (peng-robinson); T_c from the printed a(T_c,p_c)
  and b(T_c,p_c) relations in the text below that equation.
* Pseudopotential psi(rho, T), Sec. 2.1 Eq. (psi), G = -1.
* Maxwell equal-area coexistence, Sec. 3.2 (the rule the sigma tuning targets).
* Mechanical-stability coexistence integral, Sec. 3.2 Eq. (integral_coexistence_curve),
  with the sigma secant started at -16 G sigma_0 = 2.
* Planar surface tension, Sec. 3.2 Eq. (surface_tension), from the planar
  pressure-tensor balance of Sec. 2.1 (Li-Luo tensor with the (1-kappa) psi grad grad psi
  reading); kappa per mesh from Eq. (gamma-meshes-relation).
* Latent heat h_fg from the PR EOS (departure-function enthalpy), Sec. 4.2.
* Neumann solution of the one-phase Stefan problem, Sec. 4.2 Eq. (stefan-analytical).

Every integral is a library quadrature (scipy.integrate.quad) of the stated
integrand; every root is a bracketed library root finder or the secant the
paper names.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize, special

G_DEFAULT = -1.0  # Sec. 2.1, below Eq. (psi): G = -1 throughout


@dataclass(frozen=True)
class PR:
    """Peng-Robinson parameters in lattice units (Sec. 2.1, Eq. peng-robinson)."""

    a: float = 3.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    omega: float = 0.344
    G: float = G_DEFAULT

    @property
    def k(self) -> float:
        # the kappa-like factor of Eq. (peng-robinson), constants as printed
        w = self.omega
        return 0.37464 + 1.54226 * w - 0.2699 * w * w

    @property
    def Tc(self) -> float:
        # a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc  =>  Tc = 0.0778 a / (0.45724 b R)
        return 0.0778 * self.a / (0.45724 * self.b * self.R)

    def alpha(self, T):
        return (1.0 + self.k * (1.0 - np.sqrt(T / self.Tc))) ** 2

    def p(self, rho, T):
        """Eq. (peng-robinson)."""
        rho = np.asarray(rho, dtype=np.float64)
        b = self.b
        return rho * self.R * T / (1.0 - b * rho) - self.a * self.alpha(T) * rho ** 2 / (
            1.0 + 2.0 * b * rho - b * b * rho * rho)

    def dp_dT(self, rho, T):
        """(dp/dT) at constant rho, analytic derivative of Eq. (peng-robinson)."""
        rho = np.asarray(rho, dtype=np.float64)
        b, k, Tc = self.b, self.k, self.Tc
        dalpha = -k * (1.0 + k * (1.0 - np.sqrt(T / Tc))) / np.sqrt(T * Tc)
        return rho * self.R / (1.0 - b * rho) - self.a * dalpha * rho ** 2 / (
            1.0 + 2.0 * b * rho - b * b * rho * rho)

    def psi2_arg(self, rho, T):
        """Argument of the square root in Eq. (psi): 2 (p - rho/3) / G."""
        return 2.0 * (self.p(rho, T) - np.asarray(rho) / 3.0) / self.G

    def psi(self, rho, T):
        """Eq. (psi)."""
        return np.sqrt(self.psi2_arg(rho, T))


def refine_a(a_base: float, n_base: int, n: int) -> float:
    """Eq. (a-deltax): a(dx) = a_base dx^2/dx0^2 with dx proportional to 1/n."""
    return a_base * (n_base / n) ** 2


def _pressure_roots(eos: PR, T: float, p0: float):
    """Real roots in (0, 1/b) of p(rho) = p0 (the PR isotherm is a cubic in rho)."""
    a, b, R = eos.a * eos.alpha(T), eos.b, eos.R
    # p0 (1 - b r)(1 + 2 b r - b^2 r^2) = r R T (1 + 2 b r - b^2 r^2) - a r^2 (1 - b r)
    lhs = np.polynomial.Polynomial([1.0, -b]) * np.polynomial.Polynomial([1.0, 2 * b, -b * b]) * p0
    rhs = (np.polynomial.Polynomial([0.0, R * T]) * np.polynomial.Polynomial([1.0, 2 * b, -b * b])
           - np.polynomial.Polynomial([0.0, 0.0, a]) * np.polynomial.Polynomial([1.0, -b]))
    roots = (rhs - lhs).roots()
    real = sorted(r.real for r in roots if abs(r.imag) < 1e-12 * max(1.0, abs(r)) and 0 < r.real < 1 / b)
    return real


def _spinodal_pressures(eos: PR, T: float):
    """Local max and min of the sub-critical isotherm p(rho)."""
    rr = np.linspace(1e-6, 1.0 / eos.b * 0.999, 20001)
    pp = eos.p(rr, T)
    d = np.diff(pp)
    i_max = int(np.argmax(d < 0))           # first descending sample: near the local max
    i_min = i_max + int(np.argmax(d[i_max:] > 0))
    f = lambda r: -float(eos.p(r, T))
    rmax = optimize.minimize_scalar(f, bracket=(rr[max(i_max - 2, 0)], rr[i_max], rr[i_max + 2])).x
    rmin = optimize.minimize_scalar(lambda r: float(eos.p(r, T)),
                                    bracket=(rr[i_min - 2], rr[i_min], rr[i_min + 2])).x
    return float(eos.p(rmin, T)), float(eos.p(rmax, T))


def _equal_area(eos: PR, T: float, weight):
    """Solve p(rho_v) = p(rho_l) = p0 and int_{rho_v}^{rho_l} (p0 - p) weight(rho) d rho = 0."""
    p_lo, p_hi = _spinodal_pressures(eos, T)
    p_lo = max(p_lo, 1e-14)

    def g(p0):
        r = _pressure_roots(eos, T, p0)
        rv, rl = r[0], r[-1]
        val, _ = integrate.quad(lambda x: (p0 - float(eos.p(x, T))) * weight(x), rv, rl,
                                points=r[1:-1] or None, epsabs=1e-15, epsrel=1e-13, limit=400)
        return val

    eps = 1e-12 * (p_hi - p_lo)
    p0 = optimize.brentq(g, p_lo + eps, p_hi - eps, xtol=1e-16, rtol=1e-15, maxiter=500)
    r = _pressure_roots(eos, T, p0)
    return r[0], r[-1], p0


def maxwell(eos: PR, T: float):
    """Maxwell equal-area rule in the p-v plane: int (p_s - p) d(1/rho) = 0.

    Returns (rho_v, rho_l, p_sat)."""
    return _equal_area(eos, T, lambda r: 1.0 / (r * r))


def dpsi_drho(eos: PR, rho, T):
    """d psi / d rho from Eq. (psi): psi' = (dp/drho - 1/3) / (G psi)."""
    r = np.asarray(rho, dtype=np.float64)
    b, a, R = eos.b, eos.a * eos.alpha(T), eos.R
    d1 = 1.0 + 2.0 * b * r - b * b * r * r
    dp = R * T / (1.0 - b * r) ** 2 - a * (2.0 * r * d1 - r * r * (2.0 * b - 2.0 * b * b * r)) / d1 ** 2
    return (dp - 1.0 / 3.0) / (eos.G * eos.psi(r, T))


def coexistence_integral(eos: PR, T: float, sigma: float, rho_v: float, rho_l: float, p0: float):
    """Left side of Eq. (integral_coexistence_curve) with exponent 1 - 16 G sigma."""
    e = 1.0 - 16.0 * eos.G * sigma
    f = lambda r: (p0 - float(eos.p(r, T))) * float(dpsi_drho(eos, r, T)) / float(eos.psi(r, T)) ** e
    val, _ = integrate.quad(f, rho_v, rho_l, epsabs=1e-15, epsrel=1e-13, limit=400)
    return val


def mechanical_coexistence(eos: PR, T: float, sigma: float):
    """Densities selected by the mechanical-stability condition at a given sigma."""
    e = 1.0 - 16.0 * eos.G * sigma
    w = lambda r: float(dpsi_drho(eos, r, T)) / float(eos.psi(r, T)) ** e
    return _equal_area(eos, T, w)


def sigma_for(eos: PR, T: float, tol: float = 1e-13, maxit: int = 100):
    """Sec. 3.2 step 2: the sigma that puts the mechanical coexistence on the Maxwell densities.

    Secant on sigma for Eq. (integral_coexistence_curve) evaluated at the Maxwell
    (rho_v, rho_l, p_sat), started at -16 G sigma_0 = 2 (second iterate 1% away)."""
    rv, rl, ps = maxwell(eos, T)
    s0 = -2.0 / (16.0 * eos.G)
    s1 = s0 * 0.99
    f0 = coexistence_integral(eos, T, s0, rv, rl, ps)
    f1 = coexistence_integral(eos, T, s1, rv, rl, ps)
    for _ in range(maxit):
        s2 = s1 - f1 * (s1 - s0) / (f1 - f0)
        s0, f0 = s1, f1
        s1, f1 = s2, coexistence_integral(eos, T, s2, rv, rl, ps)
        if abs(s1 - s0) < tol * max(1.0, abs(s1)):
            return s1
    raise RuntimeError("sigma secant did not converge")


def planar_gamma(eos: PR, T: float, sigma: float, kappa: float):
    """Planar surface tension, Sec. 3.2 Eq. (surface_tension).

    The planar normal stress of the Sec. 2.1 pressure tensor (reading: the (1-kappa)
    term is psi grad grad psi) is P_xx = p_EOS + 2 sigma G^2 psi_x^2 + (G/4) psi psi_xx
    (c = 1), constant (= p0) across the interface. Multiplying by (8/(G psi)) psi_x psi^e,
    e = 16 G sigma, gives the first integral d(Y psi^e) = (8/(G psi)) (p0 - p_EOS) psi^e d psi
    with Y = psi_x^2, vanishing in both bulks. psi(rho) is not monotone near the liquid
    bulk, so the profile is parametrised by rho (d psi = psi'(rho) d rho) and Y psi^e is
    accumulated from the nearer bulk. Then
    gamma = (G/6)(1-kappa) int psi psi_xx dx = -(G/6)(1-kappa) int sqrt(Y) |psi'| d rho.
    """
    rv, rl, p0 = mechanical_coexistence(eos, T, sigma)
    G = eos.G
    e = 16.0 * G * sigma
    rmid = 0.5 * (rv + rl)

    def src(r):  # d(Y psi^e)/d rho along the profile
        ps = float(eos.psi(r, T))
        return (8.0 / (G * ps)) * (p0 - float(eos.p(r, T))) * ps ** e * float(dpsi_drho(eos, r, T))

    def Y(r):
        if r <= rmid:
            ye, _ = integrate.quad(src, rv, r, epsabs=1e-14, epsrel=1e-11, limit=200)
        else:
            ye, _ = integrate.quad(src, r, rl, epsabs=1e-14, epsrel=1e-11, limit=200)
            ye = -ye
        return max(ye, 0.0) * float(eos.psi(r, T)) ** (-e)

    val, _ = integrate.quad(lambda r: math.sqrt(Y(r)) * abs(float(dpsi_drho(eos, r, T))), rv, rl,
                            points=[rmid], epsabs=1e-12, epsrel=1e-9, limit=200)
    return -(G / 6.0) * (1.0 - kappa) * val


def kappa_for(eos0: PR, eos1: PR, T_ratio: float, n0: int, n1: int, sigma0: float, sigma1: float,
              kappa0: float = 0.0):
    """Sec. 3.2 step 3, Eq. (gamma-meshes-relation): gamma_1(kappa) = gamma_0 dx1/dx0.

    Reading: subscript 0 is the coarse base mesh (n0 nodes per length), 1 the finer
    one; dx is proportional to 1/n. gamma is linear in (1 - kappa), so kappa follows
    in closed form from one planar quadrature per mesh."""
    g0 = planar_gamma(eos0, T_ratio * eos0.Tc, sigma0, kappa0)
    g1_unit = planar_gamma(eos1, T_ratio * eos1.Tc, sigma1, 0.0)
    target = g0 * n0 / n1
    return 1.0 - target / g1_unit


def h_fg(eos: PR, T: float):
    """Latent heat per unit mass from the PR EOS (Sec. 4.2 names it; Gong-Cheng style).

    Enthalpy difference of the Maxwell phases with the residual (departure) internal
    energy u_res(rho) = int_0^rho (p - T dp/dT)/r^2 dr; the ideal part c_v T cancels."""
    rv, rl, ps = maxwell(eos, T)
    f = lambda r: (float(eos.p(r, T)) - T * float(eos.dp_dT(r, T))) / (r * r)
    du, _ = integrate.quad(f, rl, rv, epsabs=1e-15, epsrel=1e-13, limit=400)
    return du + ps * (1.0 / rv - 1.0 / rl)


def jakob(eos: PR, T_sat: float, dT: float, cv: float):
    """Ja = c_v (T_w - T_sat) / h_fg (Sec. 4.1 and 4.2)."""
    return cv * dT / h_fg(eos, T_sat)


def neumann_beta(ja: float):
    """Root of beta exp(beta^2) erf(beta) = Ja / sqrt(pi), Sec. 4.2."""
    f = lambda b: b * math.exp(b * b) * special.erf(b) - ja / math.sqrt(math.pi)
    return optimize.brentq(f, 1e-12, 5.0, xtol=1e-15, rtol=1e-15)


def neumann_front(beta: float, alpha_v: float, t):
    """Eq. (stefan-analytical): s(t) = 2 beta sqrt(alpha_v t)."""
    return 2.0 * beta * np.sqrt(alpha_v * np.asarray(t, dtype=np.float64))
