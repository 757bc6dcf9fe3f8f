"""GPU: the reverse-mode adjoint of the fused step (ppl_adjoint_step) with checkpointed
recomputation, for the sigma / kappa calibration of Sec. 3.2 on the lattice, at the sizes of
the calibration runs (a 256 x 8 planar interface and a 128^2 static droplet, 3,000 steps):

* against the forward-mode tangent of the same step (an independent route, FP64) to 1e-8;
* against central finite differences (h = 1e-4) of the FP64 step to 1e-5;
* against central finite differences of the FP64 oracle on a small case (tape-free FP64
  reference gradient);
* FP32 forward with FP64 accumulation against the FP64 gradient;
* the gradient does not depend on the checkpoint interval (bitwise);
* gradient descent with the autograd Function reaches the target coexistence densities."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle, thermo

pytestmark = pytest.mark.gpu

A, T_RATIO = 3.0 / 49.0, 0.86


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import calibration, ppl
    return ppl, calibration


def planar_case(C, sigma, kappa, precision, nx=256, ny=8):
    Tc, rv, rl = C._coexistence(A, T_RATIO)
    T = T_RATIO * Tc
    cfg = W.base_config(nx, ny, a=A, sigma=sigma, kappa=kappa, rho_l=rl, rho_v=rv, precision=precision,
                        rho_ref=rv, T_ref=T)
    return cfg, W.slab_fields(nx, ny, nx // 4, 3 * nx // 4, 3.0, rl, rv, T)


def droplet_case(C, sigma, kappa, precision, n=128):
    Tc, rv, rl = C._coexistence(A, T_RATIO)
    T = T_RATIO * Tc
    cfg = W.base_config(n, n, a=A, sigma=sigma, kappa=kappa, rho_l=rl, rho_v=rv, precision=precision,
                        rho_ref=rv, T_ref=T)
    return cfg, W.droplet_fields(n, n, n / 4.0, 3.0, rl, rv, T, T), (T, rv, rl)


def tangent(ppl, cfg, ic, steps, param):
    with ppl.Simulation(dict(cfg, precision="fp64_d" + param), *ic) as s:
        s.step(steps)
        return s.fields()["rho"], s.tangent_fields()["rho"]


def test_adjoint_planar_matches_tangent_and_central_differences(mods):
    ppl, C = mods
    sigma, kappa, steps = 0.11, 0.1, 3000
    cfg, ic = planar_case(C, sigma, kappa, "fp64")
    tp = C.Tape(cfg, ic, steps, interval=100)
    (rl, rv), (gl, gv) = C.planar_seed(tp.fields["rho"])
    grad_l = tp.reverse(gl)
    grad_v = tp.reverse(gv)
    tp.close()
    # kappa leaves a planar interface's densities alone (its derivative is rounding noise,
    # ~1e-9 of the sigma derivative): that component is compared on the scale of the sigma one
    for j, param in enumerate(("sigma", "kappa")):
        rho, d = tangent(ppl, cfg, ic, steps, param)
        nx = cfg["nx"]
        assert rl == pytest.approx(float(rho[:, nx // 2].mean()), rel=1e-12)
        for grad, col in ((grad_l, nx // 2), (grad_v, 0)):
            want = float(d[:, col].mean())
            assert grad[j] == pytest.approx(want, rel=1e-8, abs=1e-8 * abs(grad[0]))
    # central differences of the FP64 step
    h = 1e-4
    for j, name in enumerate(("sigma", "kappa")):
        vals = []
        for sgn in (1, -1):
            p = {"sigma": sigma, "kappa": kappa}
            p[name] += sgn * h
            c2, ic2 = planar_case(C, p["sigma"], p["kappa"], "fp64")
            with ppl.Simulation(c2, *ic2) as s:
                s.step(steps)
                vals.append(C.planar_seed(s.fields()["rho"])[0])
        fd_l = (vals[0][0] - vals[1][0]) / (2 * h)
        fd_v = (vals[0][1] - vals[1][1]) / (2 * h)
        assert grad_l[j] == pytest.approx(fd_l, rel=1e-5, abs=1e-5 * abs(grad_l[0]))
        assert grad_v[j] == pytest.approx(fd_v, rel=1e-5, abs=1e-5 * abs(grad_v[0]))


def test_adjoint_droplet_gamma_matches_tangent(mods):
    ppl, C = mods
    sigma, kappa, steps = 0.11, 0.2, 3000
    cfg, ic, (T, rv, rl) = droplet_case(C, sigma, kappa, "fp64")
    td = C.Tape(cfg, ic, steps, interval=100)
    gamma, gg = C.droplet_gamma_seed(td.fields["rho"], A, T, rv, rl)
    grad = td.reverse(gg)
    td.close()
    for j, param in enumerate(("sigma", "kappa")):
        rho, d = tangent(ppl, cfg, ic, steps, param)
        g2, dg, _ = C._droplet_gamma(rho, d, A, T, rv, rl)
        assert gamma == pytest.approx(g2, rel=1e-12)
        assert grad[j] == pytest.approx(dg, rel=1e-8)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient(mods):
    ppl, C = mods
    cfg, ic = planar_case(C, 0.11, 0.1, "fp32", nx=128, ny=4)
    grads = []
    for interval in (37, 600):
        tp = C.Tape(cfg, ic, 600, interval=interval)
        grads.append(tp.reverse(C.planar_seed(tp.fields["rho"])[1][0]))
        tp.close()
    np.testing.assert_array_equal(grads[0], grads[1])


def test_adjoint_fp32_forward_tracks_fp64(mods):
    # FP32 forward (deviation storage), FP64 adjoint and accumulation, against the FP64 sweep
    ppl, C = mods
    out = []
    for prec in ("fp64", "fp32"):
        cfg, ic = planar_case(C, 0.11, 0.1, prec)
        tp = C.Tape(cfg, ic, 3000, interval=100)
        out.append(tp.reverse(C.planar_seed(tp.fields["rho"])[1][0]))
        tp.close()
    assert out[1][0] == pytest.approx(out[0][0], rel=1e-3)
    assert abs(out[1][1] - out[0][1]) <= 1e-3 * abs(out[0][0])


def test_adjoint_against_oracle_central_differences(mods):
    # the FP64 oracle's central differences (h = 1e-4) of rho_l on a small slab: a tape-free
    # FP64 reference gradient from an implementation that shares nothing with the kernels
    ppl, C = mods
    nx, ny, steps, h = 48, 4, 400, 1e-4
    e = thermo.PR(a=A)
    T = T_RATIO * e.Tc
    rv, rl, _ = thermo.maxwell(e, T)
    base = dict(sigma=0.11, kappa=0.1)
    ic = W.slab_fields(nx, ny, nx // 4, 3 * nx // 4, 3.0, rl, rv, T)
    cfg = W.base_config(nx, ny, a=A, rho_l=rl, rho_v=rv, precision="fp64", **base)
    tp = C.Tape(cfg, ic, steps, interval=50)
    _, (gl, _) = C.planar_seed(tp.fields["rho"])
    grad = tp.reverse(gl)
    tp.close()
    for j, name in enumerate(("sigma", "kappa")):
        vals = []
        for sgn in (1, -1):
            p = dict(base)
            p[name] += sgn * h
            o = oracle.Oracle(W.base_config(nx, ny, a=A, rho_l=rl, rho_v=rv, **p), *ic)
            o.step(steps)
            vals.append(float(o.fields()["rho"][:, nx // 2].mean()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert grad[j] == pytest.approx(fd, rel=1e-5, abs=1e-5 * abs(grad[0]))


def test_adjoint_autograd_descent_to_target_densities(mods):
    # torch.autograd.Function with the adjoint backward: its gradient equals the tangent
    # route's, and gradient steps bring the planar densities to the Maxwell densities
    torch = pytest.importorskip("torch")
    ppl, C = mods
    run = dict(planar=dict(nx=128, ny=4, steps=1500), laplace=dict(n=48, R0=12.0, steps=1500))
    f_adj = C.torch_observables_adjoint(A, T_RATIO, precision="fp64", **run)
    f_tan = C.torch_observables(A, T_RATIO, **run)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    g = []
    for f in (f_adj, f_tan):
        p = torch.tensor([0.1, 0.2], dtype=torch.float64, requires_grad=True)
        (f(p) * w).sum().backward()
        g.append(p.grad.clone())
    np.testing.assert_allclose(g[0].numpy(), g[1].numpy(), rtol=1e-7)

    _, rv, rl = C._coexistence(A, T_RATIO)
    f32 = C.torch_observables_adjoint(A, T_RATIO, precision="fp32", **run)
    target = torch.tensor([rl, rv], dtype=torch.float64)
    q = torch.tensor([0.09, 0.2], dtype=torch.float64, requires_grad=True)
    losses = []
    for _ in range(5):
        q.grad = None
        obs = f32(q)
        loss = (((obs[:2] - target) / target) ** 2).sum()
        loss.backward()
        losses.append(float(loss))
        with torch.no_grad():
            gs = q.grad.clone()
            gs[1] = 0.0  # kappa leaves the planar densities alone: tune sigma
            q -= 0.5 * loss / (gs @ gs) * gs  # half a Gauss-Newton-sized step along -grad
    assert all(b < a for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.2 * losses[0]
