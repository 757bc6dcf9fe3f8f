"""Simulation-based calibration of sigma and kappa per mesh (the tuning step of Sec. 3.2),
driven by forward-mode sensitivities of the fused step (``PPL_FP64_DSIGMA`` /
``PPL_FP64_DKAPPA``).

The paper tunes sigma with a secant iteration on the coexistence integral of Eq.
(integral_coexistence_curve) and kappa with the quadrature of Eq. (surface_tension)
(``ppl_sigma_for`` / ``ppl_kappa_for``). Here the same targets are reached on the lattice
itself: sigma by Gauss-Newton on the coexistence densities of a planar interface (targets:
the Maxwell densities), kappa by Newton on the Laplace-law surface tension of a static
droplet (target: gamma of the base mesh scaled with dx, Eq. gamma-meshes-relation).
Every derivative comes from one sensitivity run on the GPU; host code forms the droplet's
radius and pressure jump from the exported fields and the Gauss-Newton step from a
handful of scalars.
"""
from __future__ import annotations

import math

import workloads as W

from . import ppl

EOS = dict(b=2.0 / 21.0, R=1.0, omega=0.344, G=-1.0)


def _coexistence(a, T_ratio):
    Tc = ppl.tc(a, EOS["b"], EOS["R"])
    rv, rl, _ = ppl.maxwell(a, EOS["b"], EOS["R"], EOS["omega"], T_ratio * Tc)
    return Tc, rv, rl


def planar_densities(a, T_ratio, sigma, nx=256, ny=8, steps=3000, width=3.0):
    """Liquid and vapour densities of a planar slab (the slab centre and the vapour centre,
    averaged across the strip) after `steps` steps, with their derivatives d/d sigma."""
    Tc, rv, rl = _coexistence(a, T_ratio)
    T = T_ratio * Tc
    cfg = W.base_config(nx, ny, a=a, sigma=sigma, rho_l=rl, rho_v=rv, precision="fp64_dsigma", T_ref=T)
    ic = W.slab_fields(nx, ny, nx // 4, 3 * nx // 4, width, rl, rv, T)
    with ppl.Simulation(cfg, *ic) as s:
        s.step(steps)
        rho = s.fields()["rho"]
        d = s.tangent_fields()["rho"]
    xl, xv = nx // 2, 0
    return (float(rho[:, xl].mean()), float(rho[:, xv].mean()), float(d[:, xl].mean()), float(d[:, xv].mean()))


def calibrate_sigma(a, T_ratio=0.86, sigma0=0.1, iters=8, tol=1e-7, **run):
    """sigma that brings the planar coexistence densities to the Maxwell densities
    (relative residuals, Gauss-Newton). Returns (sigma, history)."""
    _, rv, rl = _coexistence(a, T_ratio)
    sigma, hist = sigma0, []
    for _ in range(iters):
        ro_l, ro_v, d_l, d_v = planar_densities(a, T_ratio, sigma, **run)
        r = ((ro_l - rl) / rl, (ro_v - rv) / rv)
        J = (d_l / rl, d_v / rv)
        step = -(J[0] * r[0] + J[1] * r[1]) / (J[0] * J[0] + J[1] * J[1])
        hist.append({"sigma": sigma, "rho_l": ro_l, "rho_v": ro_v, "residual": math.hypot(*r)})
        sigma += step
        if abs(step) < tol:
            break
    return sigma, hist


def _droplet_gamma(rho, d, a, T, rv, rl):
    """gamma = (p_in - p_out) R and its derivative from a density field and its tangent.
    R = sqrt(A / pi), A the liquid fraction clamp((rho - lo) / (hi - lo), 0, 1) summed over
    the band lo, hi = rho_mid -+ 5% (rho_l - rho_v); p from the EOS at the centre (2 x 2
    mean) and at the corner node."""
    import numpy as np
    lo, hi = 0.5 * (rl + rv) - 0.05 * (rl - rv), 0.5 * (rl + rv) + 0.05 * (rl - rv)
    frac = (rho - lo) / (hi - lo)
    A = float(np.clip(frac, 0.0, 1.0).sum())
    dA = float(d[(frac > 0.0) & (frac < 1.0)].sum() / (hi - lo))
    R = math.sqrt(A / math.pi)
    dR = dA / (2.0 * math.pi * R)
    n = rho.shape[0]
    c = n // 2
    rin, din = float(rho[c - 1:c + 1, c - 1:c + 1].mean()), float(d[c - 1:c + 1, c - 1:c + 1].mean())
    rout, dout = float(rho[0, 0]), float(d[0, 0])
    pin, dpin = ppl.pressure(a, EOS["b"], EOS["R"], EOS["omega"], T, rin)
    pout, dpout = ppl.pressure(a, EOS["b"], EOS["R"], EOS["omega"], T, rout)
    dP = pin - pout
    return dP * R, (dpin * din - dpout * dout) * R + dP * dR, R


def laplace_gamma(a, T_ratio, sigma, kappa, n=128, R0=None, steps=3000, width=3.0, param="kappa"):
    """Laplace-law surface tension gamma = (p_in - p_out) R of a static droplet on an n x n
    periodic box after `steps` steps, with d gamma / d param (param: "kappa" or "sigma")."""
    Tc, rv, rl = _coexistence(a, T_ratio)
    T = T_ratio * Tc
    R0 = n / 4.0 if R0 is None else R0
    cfg = W.base_config(n, n, a=a, sigma=sigma, kappa=kappa, rho_l=rl, rho_v=rv, precision="fp64_d" + param,
                        T_ref=T)
    ic = W.droplet_fields(n, n, R0, width, rl, rv, T, T)
    with ppl.Simulation(cfg, *ic) as s:
        s.step(steps)
        rho = s.fields()["rho"]
        d = s.tangent_fields()["rho"]
    return _droplet_gamma(rho, d, a, T, rv, rl)


def calibrate_kappa(a, T_ratio, sigma, gamma_target, kappa0=0.0, iters=8, tol=1e-6, **run):
    """kappa with laplace_gamma(kappa) = gamma_target (Newton). Returns (kappa, history)."""
    kappa, hist = kappa0, []
    for _ in range(iters):
        g, dg, R = laplace_gamma(a, T_ratio, sigma, kappa, **run)
        hist.append({"kappa": kappa, "gamma": g, "R": R})
        step = -(g - gamma_target) / dg
        kappa += step
        if abs(step) < tol:
            break
    return kappa, hist


def calibrate_mesh(n_base=128, n=192, T_ratio=0.86, a_base=3.0 / 49.0, kappa_base=0.0, steps=3000):
    """Sec. 3.2 on the lattice: sigma and kappa of mesh n such that its coexistence densities
    are the Maxwell ones and its Laplace surface tension is the base mesh's times n_base / n.
    Reports the quadrature calibration (ppl_sigma_for, ppl_kappa_for) beside it."""
    r = n / n_base
    a = ppl.refine_a(a_base, n_base, n)
    sigma_b, hb = calibrate_sigma(a_base, T_ratio, steps=steps)
    gamma_b, _, _ = laplace_gamma(a_base, T_ratio, sigma_b, kappa_base, n=n_base, steps=steps)
    sigma_n, hs = calibrate_sigma(a, T_ratio, sigma0=sigma_b, steps=int(round(steps * r * r)))
    kappa_n, hk = calibrate_kappa(a, T_ratio, sigma_n, gamma_b / r, kappa0=kappa_base, n=n,
                                  steps=int(round(steps * r * r)))
    Tc = ppl.tc(a, EOS["b"], EOS["R"])
    return {
        "n_base": n_base, "n": n, "a": a,
        "sigma_base": sigma_b, "gamma_base": gamma_b, "sigma": sigma_n, "kappa": kappa_n,
        "sigma_quadrature": ppl.sigma_for(a, EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio * Tc),
        "kappa_quadrature": ppl.kappa_for(a_base, n_base, n, EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio,
                                          kappa_base),
        "history": {"sigma_base": hb, "sigma": hs, "kappa": hk},
    }


def observables(a, T_ratio, sigma, kappa, planar=None, laplace=None):
    """(rho_l, rho_v, gamma) of the planar and droplet runs and their 3 x 2 Jacobian with
    respect to (sigma, kappa), from four sensitivity runs."""
    planar = dict(planar or {})
    laplace = dict(laplace or {})
    Tc, rv, rl = _coexistence(a, T_ratio)
    T = T_ratio * Tc
    nx, ny = planar.pop("nx", 256), planar.pop("ny", 8)
    p_steps = planar.pop("steps", 3000)
    out, jac = None, [[0.0, 0.0] for _ in range(3)]
    for j, prec in enumerate(("fp64_dsigma", "fp64_dkappa")):
        cfg = W.base_config(nx, ny, a=a, sigma=sigma, kappa=kappa, rho_l=rl, rho_v=rv, precision=prec, T_ref=T)
        ic = W.slab_fields(nx, ny, nx // 4, 3 * nx // 4, 3.0, rl, rv, T)
        with ppl.Simulation(cfg, *ic) as s:
            s.step(p_steps)
            rho, d = s.fields()["rho"], s.tangent_fields()["rho"]
        vals = (float(rho[:, nx // 2].mean()), float(rho[:, 0].mean()))
        jac[0][j], jac[1][j] = float(d[:, nx // 2].mean()), float(d[:, 0].mean())
        if j == 0:
            out = list(vals)
    g, dg_dk, _ = laplace_gamma(a, T_ratio, sigma, kappa, **laplace)
    _, dg_ds, _ = laplace_gamma(a, T_ratio, sigma, kappa, param="sigma", **laplace)
    jac[2][0], jac[2][1] = dg_ds, dg_dk
    out.append(g)
    return out, jac


def torch_observables(a, T_ratio, planar=None, laplace=None):
    """A torch.autograd.Function mapping a tensor (sigma, kappa) to (rho_l, rho_v, gamma);
    its backward applies the Jacobian of the sensitivity runs (vector-Jacobian product), so
    torch optimisers can calibrate sigma and kappa by gradient descent."""
    import torch

    class _Obs(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params):
            vals, jac = observables(a, T_ratio, float(params[0]), float(params[1]), planar, laplace)
            ctx.save_for_backward(torch.tensor(jac, dtype=torch.float64))
            return torch.tensor(vals, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            (jac,) = ctx.saved_tensors
            return grad_out.to(torch.float64) @ jac

    return _Obs.apply


# ---------------------------------------------------------------------------------------
# Reverse mode: the adjoint of the fused step (ppl_adjoint_step) with checkpointed
# recomputation, so that one reverse sweep gives the derivatives of a scalar with respect to
# both parameters, whatever precision the forward run used.
# ---------------------------------------------------------------------------------------
class Tape:
    """A forward run kept for a reverse sweep: the handle, and a device snapshot of its stored
    state every `interval` steps. `fields` holds the final rho, u, T (host FP64).

    reverse(dJ_drho) runs the sweep for a scalar J of the final state that depends on it
    through rho (dJ_drho: [ny][nx]): segment by segment from the last, the segment's states
    are recomputed from its snapshot and exported in FP64, and the adjoint steps run back
    through them; d J / d(sigma, kappa) is accumulated in FP64 on the device."""

    def __init__(self, cfg: dict, ic, steps: int, interval: int = 100):
        import torch
        self.cfg = dict(cfg)
        self.steps, self.interval = int(steps), int(interval)
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self.sim = ppl.Simulation(cfg, *ic)
        # the handle's steps, its snapshots and the adjoint steps share one stream, so that
        # recomputing a segment never overwrites a tape the previous segment still reads
        self.stream = torch.cuda.Stream()
        self.sim.set_stream(self.stream)
        self.snaps = []
        done = 0
        while done < self.steps:
            buf = torch.empty(self.sim.snapshot_bytes, dtype=torch.uint8, device="cuda")
            self.sim.snapshot(buf.data_ptr())
            self.snaps.append((buf, done))
            n = min(self.interval, self.steps - done)
            self.sim.step(n)
            done += n
        self.fields = self.sim.fields()

    def reverse(self, dJ_drho):
        import numpy as np
        import torch
        nx, ny = self.nx, self.ny
        seed = np.ascontiguousarray(np.broadcast_to(np.asarray(dJ_drho, dtype=np.float64), (9, ny, nx)))
        lam = torch.from_numpy(seed).cuda()  # dJ/df_i = dJ/drho for every i (rho = sum f)
        lam2 = torch.empty_like(lam)
        grad = torch.zeros(2, dtype=torch.float64, device="cuda")
        scratch = torch.empty(ppl.adjoint_scratch_bytes(nx, ny), dtype=torch.uint8, device="cuda")
        tape_f = torch.empty((self.interval, 9, ny, nx), dtype=torch.float64, device="cuda")
        tape_T = torch.empty((self.interval, ny, nx), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        for buf, step0 in reversed(self.snaps):
            n = min(self.interval, self.steps - step0)
            self.sim.restore(buf.data_ptr(), step0)
            for m in range(n):
                self.sim.state_device(tape_f[m].data_ptr(), tape_T[m].data_ptr())
                if m + 1 < n:
                    self.sim.step(1)
            for m in reversed(range(n)):
                ppl.adjoint_step(self.cfg, tape_f[m].data_ptr(), tape_T[m].data_ptr(), lam.data_ptr(),
                                 lam2.data_ptr(), grad.data_ptr(), scratch.data_ptr(), self.stream)
                lam, lam2 = lam2, lam
        self.stream.synchronize()
        return grad.cpu().numpy()

    def close(self):
        if self.sim is not None:
            self.sim.close()
            self.sim = None
        self.snaps = []


def planar_seed(rho):
    """(rho_l, rho_v) of a planar slab (slab centre column nx/2, vapour column 0, averaged
    across the strip) and their gradients with respect to the rho field."""
    import numpy as np
    ny, nx = rho.shape
    gl, gv = np.zeros_like(rho), np.zeros_like(rho)
    gl[:, nx // 2] = 1.0 / ny
    gv[:, 0] = 1.0 / ny
    return (float(rho[:, nx // 2].mean()), float(rho[:, 0].mean())), (gl, gv)


def droplet_gamma_seed(rho, a, T, rv, rl):
    """Laplace gamma = (p_in - p_out) R of a droplet field (the measure of _droplet_gamma) and
    d gamma / d rho at every node."""
    import numpy as np
    lo, hi = 0.5 * (rl + rv) - 0.05 * (rl - rv), 0.5 * (rl + rv) + 0.05 * (rl - rv)
    frac = (rho - lo) / (hi - lo)
    A = float(np.clip(frac, 0.0, 1.0).sum())
    R = math.sqrt(A / math.pi)
    n = rho.shape[0]
    c = n // 2
    rin, rout = float(rho[c - 1:c + 1, c - 1:c + 1].mean()), float(rho[0, 0])
    pin, dpin = ppl.pressure(a, EOS["b"], EOS["R"], EOS["omega"], T, rin)
    pout, dpout = ppl.pressure(a, EOS["b"], EOS["R"], EOS["omega"], T, rout)
    dP = pin - pout
    g = np.where((frac > 0.0) & (frac < 1.0), dP / (2.0 * math.pi * R * (hi - lo)), 0.0)
    g[c - 1:c + 1, c - 1:c + 1] += 0.25 * dpin * R
    g[0, 0] -= dpout * R
    return dP * R, g


def _calibration_runs(a, T_ratio, sigma, kappa, precision, planar, laplace):
    Tc, rv, rl = _coexistence(a, T_ratio)
    T = T_ratio * Tc
    nx, ny = planar.get("nx", 256), planar.get("ny", 8)
    n = laplace.get("n", 128)
    R0 = laplace.get("R0") or n / 4.0
    cp = W.base_config(nx, ny, a=a, sigma=sigma, kappa=kappa, rho_l=rl, rho_v=rv, precision=precision,
                       rho_ref=rv, T_ref=T)
    icp = W.slab_fields(nx, ny, nx // 4, 3 * nx // 4, 3.0, rl, rv, T)
    cd = W.base_config(n, n, a=a, sigma=sigma, kappa=kappa, rho_l=rl, rho_v=rv, precision=precision, rho_ref=rv,
                       T_ref=T)
    icd = W.droplet_fields(n, n, R0, 3.0, rl, rv, T, T)
    return (cp, icp, planar.get("steps", 3000)), (cd, icd, laplace.get("steps", 3000)), (T, rv, rl)


def adjoint_observables(a, T_ratio, sigma, kappa, weights, precision="fp32", interval=100, planar=None,
                        laplace=None):
    """(rho_l, rho_v, gamma) of the planar and droplet runs and d(w . obs)/d(sigma, kappa) for
    the weights w, by two reverse sweeps (one per run) of the adjoint step."""
    (cp, icp, sp), (cd, icd, sd), (T, rv, rl) = _calibration_runs(a, T_ratio, sigma, kappa, precision,
                                                                  dict(planar or {}), dict(laplace or {}))
    tp = Tape(cp, icp, sp, interval)
    (rho_l, rho_v), (gl, gv) = planar_seed(tp.fields["rho"])
    grad = tp.reverse(weights[0] * gl + weights[1] * gv)
    tp.close()
    td = Tape(cd, icd, sd, interval)
    gamma, gg = droplet_gamma_seed(td.fields["rho"], a, T, rv, rl)
    grad = grad + td.reverse(weights[2] * gg)
    td.close()
    return [rho_l, rho_v, gamma], grad


def torch_observables_adjoint(a, T_ratio, precision="fp32", interval=100, planar=None, laplace=None):
    """torch.autograd.Function mapping (sigma, kappa) to (rho_l, rho_v, gamma) whose backward
    is the adjoint of the fused step: the forward runs (FP32 by default) keep checkpoints every
    `interval` steps, and backward() runs one reverse sweep per run for the incoming
    vector-Jacobian weights, with FP64 accumulation of the parameter gradient."""
    import torch

    class _Obs(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params):
            (cp, icp, sp), (cd, icd, sd), (T, rv, rl) = _calibration_runs(
                a, T_ratio, float(params[0]), float(params[1]), precision, dict(planar or {}), dict(laplace or {}))
            tp, td = Tape(cp, icp, sp, interval), Tape(cd, icd, sd, interval)
            (rho_l, rho_v), (gl, gv) = planar_seed(tp.fields["rho"])
            gamma, gg = droplet_gamma_seed(td.fields["rho"], a, T, rv, rl)
            ctx.tapes = (tp, td)
            ctx.seeds = (gl, gv, gg)
            return torch.tensor([rho_l, rho_v, gamma], dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            tp, td = ctx.tapes
            gl, gv, gg = ctx.seeds
            w = [float(v) for v in grad_out]
            grad = tp.reverse(w[0] * gl + w[1] * gv) + td.reverse(w[2] * gg)
            tp.close()
            td.close()
            return torch.tensor(grad, dtype=torch.float64)

    return _Obs.apply
