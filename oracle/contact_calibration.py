"""Wall density of the psi-based contact model (Eq. psi-based-formula) that gives a target
static contact angle, found with the FP64 oracle (TEST INFRASTRUCTURE: writes a workload
constant; nothing here runs on the GPU).

A droplet on the bottom wall of an isothermal box at 0.86 T_c (the contact-angle tests of
Sec. 4.3.1) relaxes for `steps` steps; its angle is read as a circular cap
(oracle.norms.contact_angle). The angle falls monotonically as rho_w grows (stronger
adhesion), so bisection on rho_w in [rho_lo, rho_hi] brackets the target.

    python -m oracle.contact_calibration [target_deg]
"""
from __future__ import annotations

import sys

import numpy as np

import workloads as W
from oracle import norms, oracle, thermo


def static_angle(rho_w: float, n: int = 80, steps: int = 12000) -> float:
    e = thermo.PR()
    rv, rl, _ = thermo.maxwell(e, 0.86 * e.Tc)
    sigma = thermo.sigma_for(e, 0.86 * e.Tc)
    cfg, ic = W.sessile_droplet(e.Tc, rv, rl, sigma, nx=n, ny=n, R0=0.2 * n, rho_w=rho_w)
    o = oracle.Oracle(cfg, *ic)
    o.step(steps)
    rho = o.fields()["rho"]
    theta = norms.contact_angle(rho, 0.5 * (rv + rl))
    if np.isnan(theta) and rho[0, :].min() > 0.5 * (rv + rl):
        return 0.0  # a liquid film over the whole wall: complete wetting
    return theta


def rho_w_for(target: float, rho_lo: float = 2.3, rho_hi: float = 6.5, tol: float = 0.5, **kw):
    t_lo, t_hi = static_angle(rho_lo, **kw), static_angle(rho_hi, **kw)
    trace = [(rho_lo, t_lo), (rho_hi, t_hi)]
    if not (t_hi <= target <= t_lo):
        raise ValueError("target %.1f deg not bracketed: %s" % (target, trace))
    for _ in range(12):
        mid = 0.5 * (rho_lo + rho_hi)
        t = static_angle(mid, **kw)
        trace.append((mid, t))
        if abs(t - target) <= tol:
            return mid, t, trace
        if t > target:
            rho_lo = mid
        else:
            rho_hi = mid
    return mid, t, trace


if __name__ == "__main__":
    target = float(sys.argv[1]) if len(sys.argv) > 1 else 60.0
    rho_w, theta, trace = rho_w_for(target)
    for r, t in trace:
        print("rho_w %.4f  theta %.2f" % (r, t))
    print("rho_w(%.1f deg) = %.4f (theta %.2f)" % (target, rho_w, theta))
