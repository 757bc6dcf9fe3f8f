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
