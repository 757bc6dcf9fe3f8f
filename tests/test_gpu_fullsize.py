"""Parity at the benchmark's full size (2048 x 4096 pool boiling, the launch configuration
bench.py times): one step from the seeded initial state is compared with the oracle on
sampled windows, each of which the oracle can compute on its own (a node depends only on
its 3-node neighbourhood; the domain-mean density is taken from the initial field).
Longer runs are checked through properties: FP32 against FP64 on the GPU."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle, thermo

pytestmark = pytest.mark.gpu

NX, NY = 2048, 4096


@pytest.fixture(scope="module")
def sim_cls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import Simulation
    return Simulation


@pytest.fixture(scope="module")
def workload():
    e = thermo.PR()
    rv, rl, _ = thermo.maxwell(e, 0.86 * e.Tc)
    return lambda prec: W.pool_boiling(e.Tc, rv, rl, 0.103, nx=NX, ny=NY, g=3e-5, precision=prec)


def windows():
    rng = np.random.default_rng(7)
    heater_x0 = (NX - int(round(0.2 * NX))) // 2
    fixed = [
        (-16, 16, 0, 24),                    # bottom wall across the periodic x seam
        (heater_x0 - 16, heater_x0 + 16, 0, 24),  # heater edge on the bottom wall
        (NX // 2 - 20, NX // 2 + 20, 0, 16),      # heater centre
        (1000, 1040, NY - 24, NY),           # top wall
        (118, 130, 100, 140),                # across a CTA strip boundary (122 columns)
        (500, 540, int(NY * 2 / 3) - 16, int(NY * 2 / 3) + 16),  # the liquid-vapour interface
    ]
    rand = []
    for _ in range(4):
        x0 = int(rng.integers(0, NX))
        y0 = int(rng.integers(3, NY - 40))
        rand.append((x0, x0 + 32, y0, y0 + 32))
    return fixed + rand


@pytest.mark.parametrize("prec,rtol,atol", [("fp64", 1e-10, 1e-13), ("fp32", 1e-5, 1e-6)])
def test_one_step_full_size_matches_oracle_windows(sim_cls, workload, prec, rtol, atol):
    # FP32 bound: seven digits of the stored deviations and about twenty rounded operations
    # between input and output of one step
    cfg, ic = workload(prec)
    sim = sim_cls(cfg, *ic)
    sim.step(1)
    f = sim.populations()
    T = sim.fields()["T"]
    sim.close()
    rbar = float(np.mean(ic[0]))
    for (x0, x1, y0, y1) in windows():
        wf, wT = oracle.window_step(cfg, ic, x0, x1, y0, y1, rbar, steps=1)
        xs = np.arange(x0, x1) % NX
        np.testing.assert_allclose(f[:, y0:y1][:, :, xs], wf, rtol=rtol, atol=atol, err_msg=str((x0, y0)))
        np.testing.assert_allclose(T[y0:y1][:, xs], wT, rtol=rtol, atol=atol * 0.1, err_msg=str((x0, y0)))


def test_full_size_fp32_tracks_fp64(sim_cls, workload):
    # 400 steps of the benchmark workload: the FP32 path stays within the FP32 budget of the
    # FP64 path in the paper's relative-difference norm (Eq. rel-diff-timestep form)
    out = {}
    for prec in ("fp64", "fp32"):
        cfg, ic = workload(prec)
        sim = sim_cls(cfg, *ic)
        sim.step(400)
        out[prec] = sim.fields()
        assert sim.norms()["flags"] == 0
        sim.close()
    for k in ("rho", "T"):
        a, b = out["fp32"][k], out["fp64"][k]
        assert np.abs(a - b).sum() / np.abs(b).sum() < 1e-5, k
