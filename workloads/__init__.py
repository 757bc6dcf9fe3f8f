"""Seeded synthetic workloads: configuration dicts and initial fields.

Shared by the CUDA path's tests and benchmark and by the CPU oracle. This module
holds geometry and parameter bookkeeping only -- no equation of state, no lattice
arithmetic. Thermodynamic inputs (T_c, coexistence densities, sigma) are passed in
by the caller, each side computing them with its own code.

Configuration dict schema (all lattice units; side order x-min, x-max, y-min, y-max):

  nx, ny                 grid size; node (x, y) is stored at [y][x]
  a, b, R, omega, G      Peng-Robinson EOS and pseudopotential strength (G < 0)
  s[9]                   MRT rates (diagonal of Lambda) in the order of M's rows
  eta_l, eta_v           kinematic viscosities; both > 0 => s[7], s[8] from eta(rho)
  rho_l, rho_v           anchors of the eta(rho) and lambda(rho) interpolations
  sigma, kappa           Li thermodynamic-consistency and surface-tension parameters
  gx, gy                 gravity (body force g (rho - rho_bar))
  cv, lambda_l, lambda_v energy equation
  energy_on, iso_steps   energy equation switch; held isothermal for the first iso_steps
  hydro_bc[4]            PERIODIC | WALL | OUTFLOW
  thermal_bc[4]          T_PERIODIC | T_DIRICHLET | T_ADIABATIC
  T_side[4], rho_w_side[4]   per-side Dirichlet temperature and wall density
  rho_w[4], T_w[4], T_dirichlet[4]   optional per-boundary-node arrays (None = per side)
  precision, rho_ref, T_ref   CUDA path only: "fp64" | "fp32"; references of the FP32
                         deviation storage f_i - w_i rho_ref and T - T_ref
"""
from __future__ import annotations

import numpy as np

PERIODIC, WALL, OUTFLOW = 0, 1, 2
T_PERIODIC, T_DIRICHLET, T_ADIABATIC = 0, 1, 2
CONTACT_PSI, CONTACT_MOD_PSI = 0, 1  # Eqs. (psi-based-formula), (mod-psi-based-formula)

# psi-based wall density of a 60 degree static contact angle at 0.86 T_c: written by
# `python -m oracle.contact_calibration 60` (FP64 oracle, 80^2 sessile drop, 12,000 steps,
# bisection on rho_w; 60.1 deg at 3.35)
RHO_W_60DEG = 3.35

# rates of the droplet/Stefan/pool runs (Sec. 4.2 and 4.3 of the paper): rho, e, zeta, j, q, j, q, eta, eta
RATES_STEFAN_POOL = [1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25]


def base_config(nx: int, ny: int, **kw) -> dict:
    cfg = dict(
        nx=int(nx), ny=int(ny),
        a=3.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344, G=-1.0,
        s=[1.0] * 9,
        eta_l=0.0, eta_v=0.0, rho_l=7.0, rho_v=0.2,
        sigma=0.0, kappa=0.0, gx=0.0, gy=0.0,
        cv=5.0, lambda_l=2.0 / 3.0, lambda_v=2.0 / 3.0,
        energy_on=0, iso_steps=0,
        hydro_bc=[PERIODIC] * 4, thermal_bc=[T_PERIODIC] * 4,
        T_side=[0.0] * 4, rho_w_side=[0.0] * 4,
        rho_w=[None] * 4, T_w=[None] * 4, T_dirichlet=[None] * 4,
        precision="fp64", rho_ref=1.0, T_ref=0.0,
        contact_model=CONTACT_PSI, G_w=0.0,
    )
    for k, v in kw.items():
        if k not in cfg:
            raise KeyError("unknown config key %r" % k)
        cfg[k] = v
    return cfg


def _tanh_profile(inside: float, outside: float, dist_inside, width: float):
    """0.5 (in + out) + 0.5 (in - out) tanh(2 d / W), d > 0 inside the region."""
    return 0.5 * (inside + outside) + 0.5 * (inside - outside) * np.tanh(2.0 * dist_inside / width)


def droplet_fields(nx, ny, R0, width, rho_in, rho_out, T_in, T_out, cx=None, cy=None):
    """Circular region of radius R0 centred in the domain (Sec. 4.1 initial profile,
    liquid inside)."""
    cx = (nx - 1) / 2.0 if cx is None else cx
    cy = (ny - 1) / 2.0 if cy is None else cy
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    rho = _tanh_profile(rho_in, rho_out, R0 - d, width)
    T = _tanh_profile(T_in, T_out, R0 - d, width)
    z = np.zeros((ny, nx))
    return rho, z.copy(), z.copy(), T


def slab_fields(nx, ny, x0, x1, width, rho_in, rho_out, T):
    """Liquid slab x0 < x < x1 across a periodic strip (planar interfaces)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.minimum(x - x0, x1 - x)
    rho = _tanh_profile(rho_in, rho_out, d, width)
    z = np.zeros((ny, nx))
    return rho, z.copy(), z.copy(), np.full((ny, nx), float(T))


def static_droplet(Tc, rho_v, rho_l, nx=64, ny=64, R0=16.0, width=3.0, T_ratio=0.8, sigma=0.1,
                   kappa=0.0, precision="fp64"):
    """Isothermal static droplet, periodic, all rates 1 (tau = 1)."""
    T = T_ratio * Tc
    cfg = base_config(nx, ny, sigma=sigma, kappa=kappa, rho_l=rho_l, rho_v=rho_v, precision=precision,
                      rho_ref=rho_v, T_ref=T)
    return cfg, droplet_fields(nx, ny, R0, width, rho_l, rho_v, T, T)


def stefan_strip(Tc, rho_v, rho_l, sigma, nx=1024, ny=4, n_vapour=10, dT_ratio=0.05, T_ratio=0.86,
                 cv=10.0, lambda_v=1.0, lambda_l=10.0, width=2.0, precision="fp64"):
    """1-D boiling-like Stefan strip (Sec. 4.2): psi-based hydrophobic wall at x = 0
    (rho_w = rho_v) held at T_sat + dT, zero-gradient outflow at x = nx-1, y periodic,
    vapour layer of n_vapour nodes, liquid at T_sat elsewhere. The FP32 storage reference is
    the liquid density: the strip is mostly liquid, whose small changes then sit in the
    low bits of near-zero deviations."""
    T_sat = T_ratio * Tc
    cfg = base_config(
        nx, ny, s=list(RATES_STEFAN_POOL), eta_l=0.1, eta_v=0.1, rho_l=rho_l, rho_v=rho_v,
        sigma=sigma, cv=cv, lambda_l=lambda_l, lambda_v=lambda_v, energy_on=1,
        hydro_bc=[WALL, OUTFLOW, PERIODIC, PERIODIC],
        thermal_bc=[T_DIRICHLET, T_ADIABATIC, T_PERIODIC, T_PERIODIC],
        T_side=[T_sat + dT_ratio * Tc, 0.0, 0.0, 0.0], rho_w_side=[rho_v, 0.0, 0.0, 0.0],
        precision=precision, rho_ref=rho_l, T_ref=T_sat)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = _tanh_profile(rho_l, rho_v, x - n_vapour, width)
    z = np.zeros((ny, nx))
    return cfg, (rho, z.copy(), z.copy(), np.full((ny, nx), T_sat))


def droplet_vaporization(Tc, rho_v, rho_l, sigma, nx=256, ny=256, R0=40.0, width=3.0, T_ratio=0.8,
                         Tv_ratio=0.9, kappa=0.3, iso_steps=10000, lam=0.25, precision="fp64"):
    """Droplet in superheated vapour (Sec. 4.1): periodic hydrodynamics, temperature held
    at T_v on the boundary ring, isothermal for the first iso_steps.

    lam: conductivity of both phases. The paper's 2/3 gives a vapour diffusivity
    lambda/(rho_v c_v) = 0.35 at T_sat = 0.86 Tc, inside the explicit Heun limit
    alpha <= 3/8 of the lattice Laplacian; at 0.8 Tc (rho_v = 0.197) it would be 0.68
    and the FD step would be unstable, hence the smaller default."""
    T_l, T_v = T_ratio * Tc, Tv_ratio * Tc
    cfg = base_config(
        nx, ny, s=[1.25] * 9, eta_l=0.1, eta_v=0.1, rho_l=rho_l, rho_v=rho_v, sigma=sigma,
        kappa=kappa, cv=5.0, lambda_l=lam, lambda_v=lam, energy_on=1, iso_steps=iso_steps,
        thermal_bc=[T_DIRICHLET] * 4, T_side=[T_v] * 4, precision=precision, rho_ref=rho_v, T_ref=T_l)
    return cfg, droplet_fields(nx, ny, R0, width, rho_l, rho_v, T_l, T_v)


def pool_boiling(Tc, rho_v, rho_l, sigma, nx=1024, ny=2048, g=3e-5, g_ref_height=160, T_ratio=0.86,
                 heater_frac=0.2,
                 dTh_ratio=0.1, rho_w_heater=RHO_W_60DEG, rho_w_bottom=RHO_W_60DEG, rho_w_top=0.38,
                 pool_frac=2.0 / 3.0, noise_ratio=1e-3, seed=20220112, width=3.0, precision="fp64"):
    """2-D pool boiling (Sec. 4.3): x periodic, Zou-He walls at y = 0 and y = ny-1,
    bottom-centre heater strip of heater_frac * nx nodes held at T_sat + dTh (Dirichlet),
    adiabatic elsewhere; psi-based wall densities per wall node (a 60 degree contact angle on
    the bottom wall and the heater, hydrophobic top); liquid pool below
    pool_frac * ny at T_sat with seeded uniform noise of +-noise_ratio * Tc.

    Gravity: g is the acceleration of a pool g_ref_height nodes tall (the paper's 160^2
    base mesh); taller grids get g * g_ref_height / ny, which keeps the hydrostatic head
    rho_l g H (~0.75 p_sat) of that pool. Without it a 4096-node column at g = 3e-5 would
    carry ~20 p_sat and push the liquid out of the EOS's domain near the bottom."""
    T_sat = T_ratio * Tc
    g = g * min(1.0, g_ref_height / float(ny))
    T_h = T_sat + dTh_ratio * Tc
    w = max(1, int(round(heater_frac * nx)))
    x0 = (nx - w) // 2
    heater = np.zeros(nx, dtype=np.uint8)
    heater[x0:x0 + w] = 1
    rho_w_b = np.where(heater == 1, rho_w_heater, rho_w_bottom).astype(np.float64)
    T_w_b = np.where(heater == 1, T_h, T_sat).astype(np.float64)
    cfg = base_config(
        nx, ny, s=list(RATES_STEFAN_POOL), eta_l=0.1, eta_v=0.1, rho_l=rho_l, rho_v=rho_v,
        sigma=sigma, gx=0.0, gy=-g, cv=5.0, lambda_l=1.95, lambda_v=0.114, energy_on=1,
        hydro_bc=[PERIODIC, PERIODIC, WALL, WALL],
        thermal_bc=[T_PERIODIC, T_PERIODIC, T_ADIABATIC, T_ADIABATIC],
        T_side=[0.0, 0.0, T_sat, T_sat], rho_w_side=[0.0, 0.0, rho_w_bottom, rho_w_top],
        rho_w=[None, None, rho_w_b, None], T_w=[None, None, T_w_b, None],
        T_dirichlet=[None, None, heater, None], precision=precision, rho_ref=rho_v, T_ref=T_sat)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = _tanh_profile(rho_l, rho_v, pool_frac * ny - y, width)
    rng = np.random.default_rng(seed)
    T = T_sat + noise_ratio * Tc * rng.uniform(-1.0, 1.0, size=(ny, nx))
    z = np.zeros((ny, nx))
    return cfg, (rho, z.copy(), z.copy(), T)


def random_smooth_density(nx, ny, rho_lo, rho_hi, seed, modes=3):
    """Smooth periodic random density field in [rho_lo, rho_hi] (a few Fourier modes)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    acc = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(1, 3, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        acc += np.cos(2 * np.pi * kx * x / nx + ph[0]) * np.cos(2 * np.pi * ky * y / ny + ph[1])
    acc = (acc - acc.min()) / (acc.max() - acc.min())
    return rho_lo + (rho_hi - rho_lo) * acc


def sessile_droplet(Tc, rho_v, rho_l, sigma, nx=160, ny=160, R0=None, width=3.0, T_ratio=0.86,
                    contact_model=CONTACT_PSI, rho_w=4.0, G_w=-0.8, rho_w_top=None, precision="fp64"):
    """Contact-angle test of Sec. 4.3.1: isothermal droplet initialised on the bottom wall
    (centre one radius above it, so that it touches the wall), x periodic, Zou-He walls at
    y = 0 and y = ny-1, the pool-boiling rates, eta = 0.1. contact_model CONTACT_PSI uses
    rho_w at the bottom wall (Eq. psi-based-formula; the top wall holds rho_w_top, default
    rho_v); CONTACT_MOD_PSI uses G_w on both walls (Eq. mod-psi-based-formula)."""
    T = T_ratio * Tc
    R0 = nx / 5.0 if R0 is None else R0
    cfg = base_config(
        nx, ny, s=list(RATES_STEFAN_POOL), eta_l=0.1, eta_v=0.1, rho_l=rho_l, rho_v=rho_v, sigma=sigma,
        hydro_bc=[PERIODIC, PERIODIC, WALL, WALL],
        thermal_bc=[T_PERIODIC, T_PERIODIC, T_ADIABATIC, T_ADIABATIC], T_side=[0.0, 0.0, T, T],
        rho_w_side=[0.0, 0.0, rho_w, rho_v if rho_w_top is None else rho_w_top],
        contact_model=contact_model, G_w=G_w, precision=precision, rho_ref=rho_v, T_ref=T)
    return cfg, droplet_fields(nx, ny, R0, width, rho_l, rho_v, T, T, cx=(nx - 1) / 2.0, cy=R0)


def paper_pool_boiling(Tc, rho_v, rho_l, sigma, n=160, rho_wh=3.44, Th_ratio=1.2, g=2.5e-5, heater_frac=0.2,
                       width=None, precision="fp64", per_node=True):
    """Pool boiling with the settings of the paper's refinement study (Sec. 4.3.2): n x n, x
    periodic, Zou-He walls at y = 0 and y = n-1, both walls held at T_sat = 0.86 T_c except
    the bottom-centre heater (heater_frac of the width) at Th_ratio T_c; rho_w 6.50 on the
    bottom wall, rho_wh on the heater, 0.38 on the top wall; liquid below half height at
    T_sat, at rest; gravity -g along y; c_v = 5, lambda 1.95 / 0.114, eta = 0.1, the
    pool-boiling rates. per_node=False leaves out the heater's per-node arrays (a
    prototype for ppl_refine, which rescales only per-side values)."""
    T_sat = 0.86 * Tc
    width = 3.0 * n / 160.0 if width is None else width
    w = max(1, int(round(heater_frac * n)))
    x0 = (n - w) // 2
    heater = np.zeros(n, dtype=bool)
    heater[x0:x0 + w] = True
    cfg = base_config(
        n, n, s=list(RATES_STEFAN_POOL), eta_l=0.1, eta_v=0.1, rho_l=rho_l, rho_v=rho_v, sigma=sigma,
        gy=-g, cv=5.0, lambda_l=1.95, lambda_v=0.114, energy_on=1,
        hydro_bc=[PERIODIC, PERIODIC, WALL, WALL],
        thermal_bc=[T_PERIODIC, T_PERIODIC, T_DIRICHLET, T_DIRICHLET],
        T_side=[0.0, 0.0, T_sat, T_sat], rho_w_side=[0.0, 0.0, 6.50, 0.38],
        precision=precision, rho_ref=rho_v, T_ref=T_sat)
    if per_node:
        cfg["rho_w"] = [None, None, np.where(heater, rho_wh, 6.50).astype(np.float64), None]
        cfg["T_w"] = [None, None, np.where(heater, Th_ratio * Tc, T_sat).astype(np.float64), None]
    y, _ = np.mgrid[0:n, 0:n].astype(np.float64)
    rho = _tanh_profile(rho_l, rho_v, 0.5 * n - y, width)
    z = np.zeros((n, n))
    T = np.full((n, n), T_sat)
    T[0, heater] = Th_ratio * Tc
    return cfg, (rho, z.copy(), z.copy(), T)
