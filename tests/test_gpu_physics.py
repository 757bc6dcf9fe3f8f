"""GPU: physics checks of the fused step on the paper's test problems.

* Stefan strip (Sec. 4.2, Eq. stefan-analytical), 1024 x 4 at the workload's settings, FP64,
  200,000 steps: the front against Neumann's s(t) = 2 beta sqrt(alpha_v t). The model is
  compressible (the paper: the LBM need not converge to this reference), the front lags it
  while the strip's pressure relaxes; the lag shrinks and the late growth exponent tends to
  Neumann's 1/2 from above.
* Droplet vaporization (Sec. 4.1): R^2(t) linear in time over the evaporation phase (the
  D^2 law), on one mesh and on the refinement batch 128^2 / 256^2 / 512^2 (1 : 4 : 16 steps
  per coarse step), whose two finer meshes agree on the slope."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import thermo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import ppl as mod
    return mod


def test_stefan_front_approaches_neumann(ppl):
    e = thermo.PR()
    Tc, Tsat = e.Tc, 0.86 * e.Tc
    rv, rl, _ = thermo.maxwell(e, Tsat)
    cfg, ic = W.stefan_strip(Tc, rv, rl, thermo.sigma_for(e, Tsat), nx=1024, ny=4, n_vapour=10)
    beta = thermo.neumann_beta(thermo.jakob(e, Tsat, cfg["T_side"][0] - Tsat, cfg["cv"]))
    alpha_v = cfg["lambda_v"] / (rv * cfg["cv"])
    t0 = (10.0 / (2.0 * beta)) ** 2 / alpha_v
    mid = 0.5 * (rv + rl)
    t, s, Ti = [], [], []
    with ppl.Simulation(cfg, *ic) as sim:
        for k in range(20):
            sim.step(10000)
            fl = sim.fields()
            p = fl["rho"].mean(axis=0)
            i = int(np.argmax(p > mid))
            x = i - 1 + (mid - p[i - 1]) / (p[i] - p[i - 1])
            t.append((k + 1) * 10000.0)
            s.append(x)
            Ti.append(float(np.interp(x, np.arange(p.size), fl["T"].mean(axis=0))))
        assert sim.norms()["flags"] == 0
    t, s = np.array(t), np.array(s)
    ratio = s / thermo.neumann_front(beta, alpha_v, t + t0)
    assert np.all(np.diff(s) > 0)
    assert np.all(np.diff(ratio[9:]) > 0)  # the lag shrinks over the second half
    assert 0.8 <= ratio[-1] <= 1.0
    k = np.polyfit(np.log(t[9:] + t0), np.log(s[9:]), 1)[0]
    assert 0.5 < k < 0.6  # growth exponent, Neumann's 1/2 approached from above
    assert all(x > Tsat for x in Ti) and Ti[-1] < Ti[9]


def _linear_fit(t, r2):
    A, B = np.polyfit(t, r2, 1)
    res = r2 - (A * t + B)
    return A, float(np.sqrt((res ** 2).mean()) / np.ptp(r2))


def test_d2_law_single_mesh(ppl):
    # 96^2, droplet R0 = 15 at 0.8 T_c in vapour held at 0.95 T_c (kappa 0.3, lambda 0.25): the
    # droplet evaporates within 250,000 steps; over the evaporation phase (R^2 from 90 % to
    # 30 % of its largest value) R^2 is linear in t to a residual of 3 % of its range
    e = thermo.PR()
    rv, rl, _ = thermo.maxwell(e, 0.8 * e.Tc)
    sig = thermo.sigma_for(e, 0.8 * e.Tc)
    cfg, ic = W.droplet_vaporization(e.Tc, rv, rl, sig, nx=96, ny=96, R0=15.0, Tv_ratio=0.95, iso_steps=10000,
                                     precision="fp32")
    mid, band = 0.5 * (rv + rl), 0.05 * (rl - rv)
    t, R = [], []
    with ppl.Simulation(cfg, *ic) as sim:
        for k in range(64):
            sim.step(4000)
            t.append((k + 1) * 4000.0)
            R.append(math.sqrt(sim.phase_area(mid - band, mid + band) / math.pi))
        assert sim.norms()["flags"] == 0
    t, r2 = np.array(t), np.array(R) ** 2
    top = int(np.argmax(r2))
    sel = (np.arange(t.size) > top) & (r2 < 0.9 * r2[top]) & (r2 > 0.3 * r2[top])
    assert sel.sum() >= 20
    slope, resid = _linear_fit(t[sel], r2[sel])
    assert slope < 0
    assert resid <= 0.03
    assert R[-1] < 0.5 * R[0]


def test_d2_law_refinement_batch(ppl):
    # the refinement sequence of the droplet-vaporization case (128^2 / 256^2 / 512^2, R = 20
    # on 128^2, 1 : 4 : 16 steps per coarse step, 200,000 coarse steps): on every mesh R^2 is
    # linear over the evaporation phase (residual 5 % of its range), the slopes (in coarse units)
    # are negative, the two finer meshes agree within 5 %, and refining moves the slope less
    # each time
    from paper_2201_04560_gb300 import refinement
    out = refinement.droplet_vaporization_study(meshes=(128, 256, 512), R0=20.0, coarse_steps=200000,
                                                sample_every=2000)
    t = np.asarray(out["t"], dtype=np.float64)
    slopes = []
    for R in out["R"]:
        r2 = np.asarray(R) ** 2
        sel = (t > 10000) & (r2 > 0.25 * 400.0)
        slope, resid = _linear_fit(t[sel], r2[sel])
        assert resid <= 0.05
        slopes.append(slope)
    assert all(s < 0 for s in slopes)
    assert abs(slopes[2] - slopes[1]) <= 0.05 * abs(slopes[2])
    assert abs(slopes[2] - slopes[1]) < abs(slopes[1] - slopes[0])
