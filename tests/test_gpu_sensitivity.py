"""GPU: forward-mode sensitivities of the fused step with respect to sigma (Eq. S) and kappa
(Eq. Q) through the C ABI, against central finite differences of the FP64 step (h = 1e-4)
and against Richardson-extrapolated central differences of the FP64 oracle; the value part
of a sensitivity run against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle, thermo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import ppl as mod
    return mod


@pytest.fixture(scope="module")
def th():
    e = thermo.PR()
    return {"e": e, 0.8: thermo.maxwell(e, 0.8 * e.Tc), 0.86: thermo.maxwell(e, 0.86 * e.Tc)}


def make_case(th, name):
    e = th["e"]
    if name == "droplet":
        rv, rl, _ = th[0.8]
        cfg, ic = W.static_droplet(e.Tc, rv, rl, nx=48, ny=44, R0=11.0, kappa=0.2)
        return cfg, ic, 300
    if name == "vaporization":
        rv, rl, _ = th[0.8]
        cfg, ic = W.droplet_vaporization(e.Tc, rv, rl, 0.1, nx=40, ny=40, R0=10.0, iso_steps=20)
        return cfg, ic, 150
    rv, rl, _ = th[0.86]
    cfg, ic = W.pool_boiling(e.Tc, rv, rl, 0.1032, nx=48, ny=40, g=3e-5)
    cfg.update(kappa=0.15)
    return cfg, ic, 120


def run(ppl, cfg, ic, steps, **over):
    c = dict(cfg, **over)
    with ppl.Simulation(c, *ic) as s:
        s.step(steps)
        out = s.fields()
        if "_d" in c.get("precision", "fp64"):
            out["d"] = s.tangent_fields()
    return out


def rel_inf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", ["droplet", "vaporization", "pool"])
@pytest.mark.parametrize("param", ["sigma", "kappa"])
def test_tangent_matches_central_differences(ppl, th, name, param):
    cfg, ic, steps = make_case(th, name)
    # central differences with h = 1e-4 carry an O(h^2) truncation error (up to ~2e-5 of
    # the derivative in the pool case); their Richardson extrapolation with h / 2 removes
    # it, and the tangent must agree with that to 1e-6
    tan = run(ppl, cfg, ic, steps, precision="fp64_d" + param)
    h = 1e-4
    p0 = cfg[param]
    D = {}
    for hh in (h, h / 2):
        plus = run(ppl, cfg, ic, steps, **{param: p0 + hh})
        minus = run(ppl, cfg, ic, steps, **{param: p0 - hh})
        D[hh] = {f: (plus[f] - minus[f]) / (2 * hh) for f in ("rho", "T", "ux", "uy")}
    for f in ("rho", "T", "ux", "uy"):
        fd = D[h][f]
        if np.max(np.abs(fd)) < 1e-9 and f != "rho":
            assert np.max(np.abs(tan["d"][f])) < 1e-8  # e.g. T frozen in the isothermal phase
            continue
        assert rel_inf(tan["d"][f], fd) <= 1e-4, (f, rel_inf(tan["d"][f], fd))
        rich = (4 * D[h / 2][f] - D[h][f]) / 3
        assert rel_inf(tan["d"][f], rich) <= 1e-6, (f, rel_inf(tan["d"][f], rich))
    assert np.max(np.abs(tan["d"]["rho"])) > 1e-6  # the parameter does act on the state


@pytest.mark.parametrize("param", ["sigma", "kappa"])
def test_tangent_values_and_oracle_gradient(ppl, th, param):
    # value part: the FP64 step (oracle parity bound); derivative: Richardson extrapolation
    # (4 D(h/2) - D(h)) / 3 of the oracle's central differences, error O(h^4)
    cfg, ic, _ = make_case(th, "vaporization")
    steps = 60
    tan = run(ppl, cfg, ic, steps, precision="fp64_d" + param)

    def orc(p):
        o = oracle.Oracle(dict(cfg, **{param: p}), *ic)
        o.step(steps)
        return o.fields()

    want = orc(cfg[param])
    assert rel_inf(tan["rho"], want["rho"]) <= 1e-10
    assert rel_inf(tan["T"], want["T"]) <= 1e-10
    p0, h = cfg[param], 2e-3
    D = {}
    for hh in (h, h / 2):
        a, b = orc(p0 + hh), orc(p0 - hh)
        D[hh] = {f: (a[f] - b[f]) / (2 * hh) for f in ("rho", "T", "ux")}
    for f in ("rho", "T", "ux"):
        ref = (4 * D[h / 2][f] - D[h][f]) / 3
        assert rel_inf(tan["d"][f], ref) <= 1e-7, (f, rel_inf(tan["d"][f], ref))


def test_tangent_mode_rejected_where_unsupported(ppl, th):
    cfg, ic, _ = make_case(th, "droplet")
    with ppl.Simulation(dict(cfg, precision="fp64_dsigma"), *ic) as s, ppl.Simulation(cfg, *ic) as plain:
        with pytest.raises(ppl.PplError):
            ppl.cross_norm(s, plain, "rho")
        with pytest.raises(ppl.PplError):
            s.wall_heat_flux(2)
        assert s.phase_area(0.2, 6.0) == pytest.approx(plain.phase_area(0.2, 6.0), rel=1e-13)
        with pytest.raises(ppl.PplError):
            plain.tangent_fields()


def test_sigma_calibration_reaches_maxwell_densities(ppl):
    # Gauss-Newton on the planar coexistence densities (sensitivities d rho / d sigma)
    from paper_2201_04560_gb300 import calibration as C
    a = 3.0 / 49.0
    sigma, hist = C.calibrate_sigma(a, 0.86, sigma0=0.08, steps=3000)
    assert hist[-1]["residual"] < 2e-3
    assert hist[-1]["residual"] < 0.2 * hist[0]["residual"]
    quad = ppl.sigma_for(a, 2 / 21, 1.0, 0.344, -1.0, 0.86 * ppl.tc(a, 2 / 21, 1.0))
    assert sigma == pytest.approx(quad, rel=0.1)  # lattice vs continuum calibration of Eq. S


def test_kappa_calibration_recovers_a_known_kappa(ppl):
    # Newton on the Laplace-law surface tension (sensitivities d rho / d kappa): the gamma
    # measured at kappa = 0.3 is reached again from kappa = 0
    from paper_2201_04560_gb300 import calibration as C
    a, T_ratio = 3.0 / 49.0, 0.86
    sigma = ppl.sigma_for(a, 2 / 21, 1.0, 0.344, -1.0, T_ratio * ppl.tc(a, 2 / 21, 1.0))
    run = dict(n=64, R0=16.0, steps=2000)
    g_target, dg, _ = C.laplace_gamma(a, T_ratio, sigma, 0.3, **run)
    assert dg < 0  # (1 - kappa) scaling of gamma
    kappa, hist = C.calibrate_kappa(a, T_ratio, sigma, g_target, kappa0=0.0, **run)
    assert kappa == pytest.approx(0.3, abs=2e-3)


def test_autograd_function_gradient_and_descent(ppl):
    # the torch.autograd.Function over (sigma, kappa) -> (rho_l, rho_v, gamma): its
    # vector-Jacobian product against central differences of the observables (h = 1e-4),
    # and one gradient step on a calibration loss lowers it
    torch = pytest.importorskip("torch")
    from paper_2201_04560_gb300 import calibration as C
    a, T_ratio = 3.0 / 49.0, 0.86
    run = dict(planar=dict(nx=128, ny=4, steps=1500), laplace=dict(n=48, R0=12.0, steps=1500))
    f = C.torch_observables(a, T_ratio, **run)
    p = torch.tensor([0.1, 0.2], dtype=torch.float64, requires_grad=True)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (f(p) * w).sum().backward()
    h = 1e-4
    for i in range(2):
        hp = [0.1, 0.2]
        hm = [0.1, 0.2]
        hp[i] += h
        hm[i] -= h
        yp, _ = C.observables(a, T_ratio, *hp, **run)
        ym, _ = C.observables(a, T_ratio, *hm, **run)
        fd = sum(wi * (u - v) / (2 * h) for wi, u, v in zip(w.tolist(), yp, ym))
        assert float(p.grad[i]) == pytest.approx(fd, rel=1e-4)

    _, rv, rl = C._coexistence(a, T_ratio)
    target = torch.tensor([rl, rv, 0.9 * float(f(p.detach())[2])], dtype=torch.float64)

    def loss(q):
        return (((f(q) - target) / target) ** 2).sum()

    q = torch.tensor([0.1, 0.2], dtype=torch.float64, requires_grad=True)
    L0 = loss(q)
    L0.backward()
    with torch.no_grad():
        g = q.grad
        q2 = q - 0.5 * L0 / (g @ g) * g  # half a Gauss-Newton-sized step along -grad
    assert float(loss(q2)) < float(L0)


@pytest.mark.parametrize("name", ["droplet", "vaporization", "pool"])
@pytest.mark.parametrize("param", ["sigma", "kappa"])
def test_fp32_tangent_tracks_fp64_tangent(ppl, th, name, param):
    # FP32 forward (deviation storage, FP64 domain sums) against the FP64 sensitivity run:
    # values within the FP32 budget, derivatives within 1e-3 in the L1 norm of the field
    cfg, ic, steps = make_case(th, name)
    t64 = run(ppl, cfg, ic, steps, precision="fp64_d" + param)
    t32 = run(ppl, cfg, ic, steps, precision="fp32_d" + param)
    for f in ("rho", "T"):
        assert float(np.abs(t32[f] - t64[f]).sum() / np.abs(t64[f]).sum()) <= 1e-4
    for f in ("rho", "ux", "uy"):
        ref = t64["d"][f]
        assert float(np.abs(t32["d"][f] - ref).sum() / np.abs(ref).sum()) <= 1e-3, f
