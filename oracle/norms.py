"""Cross-mesh differences of Sec. 4.3, Eqs. (rel-diff-timestep) and (global-rel-diff).

TEST INFRASTRUCTURE ONLY: only tests/ and the CPU legs of bench.py use it.

d^N theta(t) compares a field on mesh N with the same field on the next finer mesh N*:
the coarse field is interpolated linearly onto the fine nodes (I(theta^N)) and the L1
norm of the difference over the fine nodes is divided by the L1 norm of the fine field.
D^N theta sums numerator and denominator over the output times as well.

Reading of "interpolating linearly" on a 2D mesh: bilinear in physical position. A node's
position on a mesh of n nodes over a length L is (g + 1/2) L / n on a periodic axis (the
nodes are cell centres of a torus) and g L / (n - 1) on a bounded axis (the first and last
nodes sit on the two walls). The interpolation itself is scipy's RegularGridInterpolator
(method "linear"); periodic axes are extended by one wrapped node on each side first.
"""
from __future__ import annotations

import numpy as np
from scipy.interpolate import RegularGridInterpolator


def positions(n: int, periodic: bool, length: float = 1.0) -> np.ndarray:
    """Physical coordinates of the n nodes of one axis."""
    g = np.arange(n, dtype=np.float64)
    if periodic:
        return (g + 0.5) * length / n
    return g * length / (n - 1) if n > 1 else np.zeros(1)


def interpolate(coarse: np.ndarray, fine_shape, periodic_x: bool, periodic_y: bool) -> np.ndarray:
    """I(theta^N): the coarse field [ny_c][nx_c] evaluated bilinearly at the fine nodes."""
    coarse = np.asarray(coarse, dtype=np.float64)
    nyc, nxc = coarse.shape
    nyf, nxf = fine_shape
    xc, yc = positions(nxc, periodic_x), positions(nyc, periodic_y)
    vals = coarse
    if periodic_x:  # one wrapped node on each side of the torus
        xc = np.concatenate(([xc[0] - 1.0 / nxc], xc, [xc[-1] + 1.0 / nxc]))
        vals = np.concatenate((vals[:, -1:], vals, vals[:, :1]), axis=1)
    if periodic_y:
        yc = np.concatenate(([yc[0] - 1.0 / nyc], yc, [yc[-1] + 1.0 / nyc]))
        vals = np.concatenate((vals[-1:, :], vals, vals[:1, :]), axis=0)
    if len(xc) == 1:  # a single node: constant along that axis
        xc = np.array([0.0, 1.0])
        vals = np.concatenate((vals, vals), axis=1)
    if len(yc) == 1:
        yc = np.array([0.0, 1.0])
        vals = np.concatenate((vals, vals), axis=0)
    interp = RegularGridInterpolator((yc, xc), vals, method="linear", bounds_error=False, fill_value=None)
    xf, yf = positions(nxf, periodic_x), positions(nyf, periodic_y)
    Y, X = np.meshgrid(yf, xf, indexing="ij")
    return interp(np.stack((Y.ravel(), X.ravel()), axis=1)).reshape(nyf, nxf)


def rel_diff_terms(coarse, fine, periodic_x: bool, periodic_y: bool):
    """Numerator and denominator of Eq. (rel-diff-timestep) at one time."""
    fine = np.asarray(fine, dtype=np.float64)
    I = interpolate(coarse, fine.shape, periodic_x, periodic_y)
    return float(np.sum(np.abs(I - fine))), float(np.sum(np.abs(fine)))


def rel_diff(coarse, fine, periodic_x: bool, periodic_y: bool) -> float:
    """d^N theta(t), Eq. (rel-diff-timestep)."""
    num, den = rel_diff_terms(coarse, fine, periodic_x, periodic_y)
    return num / den


def global_rel_diff(pairs, periodic_x: bool, periodic_y: bool) -> float:
    """D^N theta, Eq. (global-rel-diff): pairs = [(coarse_k, fine_k)] over output times t_k."""
    terms = [rel_diff_terms(c, f, periodic_x, periodic_y) for c, f in pairs]
    return sum(t[0] for t in terms) / sum(t[1] for t in terms)


def convergence_order(D_coarse: float, D_fine: float, h_coarse: float, h_fine: float) -> float:
    """Observed order p of D ~ h^p between two successive mesh pairs."""
    return float(np.log(D_coarse / D_fine) / np.log(h_coarse / h_fine))


def phase_area(rho, rho_lo: float, rho_hi: float) -> float:
    """Liquid area in nodes (Sec. 4.1 droplet radius R = sqrt(area / pi)): the sum of the
    liquid volume fraction clamp((rho - rho_lo) / (rho_hi - rho_lo), 0, 1)."""
    frac = (np.asarray(rho, dtype=np.float64) - rho_lo) / (rho_hi - rho_lo)
    return float(np.sum(np.clip(frac, 0.0, 1.0)))


def relative_change_R(R, R_star) -> float:
    """Eq. (relative-change-R): sum_t |R(t) - R*(t)| / sum_t |R*(t)|."""
    R, R_star = np.asarray(R, dtype=np.float64), np.asarray(R_star, dtype=np.float64)
    return float(np.sum(np.abs(R - R_star)) / np.sum(np.abs(R_star)))


def wall_heat_flux(rho, T, side: int, rho_v: float, rho_l: float, lambda_v: float, lambda_l: float) -> float:
    """Eq. (pool-heat-flux): mean over boundary line `side` (0 x-min, 1 x-max, 2 y-min,
    3 y-max) of -lambda(rho) dT/dn, n the inward normal. The derivative is the second-order
    one-sided difference (-3 T_0 + 4 T_1 - T_2) / 2 over the line and the next two inward;
    lambda(rho) is the linear law of the energy equation. Positive when heat enters."""
    rho, T = np.asarray(rho, dtype=np.float64), np.asarray(T, dtype=np.float64)
    # bring the side to row 0 with the inward direction along +rows
    if side == 2:
        r, t = rho, T
    elif side == 3:
        r, t = rho[::-1, :], T[::-1, :]
    elif side == 0:
        r, t = rho.T, T.T
    else:
        r, t = rho.T[::-1, :], T.T[::-1, :]
    lam = lambda_v + (lambda_l - lambda_v) * (r[0] - rho_v) / (rho_l - rho_v)
    dTdn = 0.5 * (-3.0 * t[0] + 4.0 * t[1] - t[2])
    return float(np.mean(-lam * dTdn))


def _crossing(values, level):
    """Fractional index where a 1-D profile first crosses `level` from above (linear)."""
    v = np.asarray(values, dtype=np.float64)
    for i in range(len(v) - 1):
        if (v[i] - level) * (v[i + 1] - level) <= 0.0 and v[i] != v[i + 1]:
            return i + (v[i] - level) / (v[i] - v[i + 1])
    return float("nan")


def contact_angle(rho, rho_mid: float) -> float:
    """Contact angle (degrees, through the liquid) of one droplet sitting on the wall line
    y = 0 of a density field [ny][nx], read as a circular cap. The base is taken on the
    first line y0 (from the wall inward, below half height) whose densest node exceeds
    rho_mid with a crossing of rho = rho_mid on each side of it (a density layer at the
    wall can hide the foot on the wall line itself); its half-width a comes from the two
    crossings, the top h from the crossing along the column through the base centre. The
    circle through (+-a, y0) and (0, h) has radius Rc = (a^2 + (h - y0)^2) / (2 (h - y0))
    and centre height yc = h - Rc; theta = 90 deg + asin(yc / Rc), clamped to [0, 180] (a
    droplet that left the wall reads 180). NaN if no base is found (e.g. a film over the
    whole wall)."""
    rho = np.asarray(rho, dtype=np.float64)
    ny = rho.shape[0]
    for y0 in range(ny // 2):
        line = rho[y0, :]
        cx = int(np.argmax(line))
        if line[cx] <= rho_mid:
            continue
        right = cx + _crossing(line[cx:], rho_mid)
        left = cx - _crossing(line[cx::-1], rho_mid)
        if not (np.isfinite(right) and np.isfinite(left)):
            continue
        a = 0.5 * (right - left)
        centre = int(round(0.5 * (right + left)))
        h = y0 + _crossing(rho[y0:, centre], rho_mid)
        if not np.isfinite(h) or h <= y0:
            return float("nan")
        Rc = (a * a + (h - y0) ** 2) / (2.0 * (h - y0))
        yc = h - Rc
        return float(90.0 + np.degrees(np.arcsin(np.clip(yc / Rc, -1.0, 1.0))))
    return float("nan")
