"""Mesh-refinement studies of Secs. 3-4, driven entirely through the C ABI.

Each study builds the problem on a sequence of meshes with the refinement procedure of
Sec. 3 (``ppl_refine``: a ~ dx^2, T ~ T_c, g ~ dx^3, sigma and kappa re-tuned per mesh,
dt ~ dx^2), advances all meshes together as one batch (``ppl_batch_*``: mesh k takes
(n_k / n_0)^2 steps per coarse step, the grids run as concurrent branches of one CUDA
graph, each with its autotuned launch shape) and evaluates the paper's cross-mesh
measures with the library's reductions: the droplet radius R(t) and Eq. (relative-change-R)
(Sec. 4.1, Table 2), the contact angle and the relative change of the density fields
(Sec. 4.3.1), the space-time differences d^N and D^N of Eqs. (rel-diff-timestep) and
(global-rel-diff), the heat flux Q(t) of Eq. (pool-heat-flux) and the time shift of
Eq. (rel-diff-minimize) (Sec. 4.3.2). Host code here only schedules calls and converts
units (lengths and times to the coarsest mesh's).
"""
from __future__ import annotations

import math
import time
from fractions import Fraction

import numpy as np

import workloads as W

from . import ppl

# Peng-Robinson constants of the paper's base mesh (Sec. 3.2, reading a = 3/49)
EOS = dict(a=3.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344, G=-1.0)


def substeps(meshes, base):
    """Smallest integer steps per outer step with dt ~ dx^2: mesh n takes (n / base)^2 times
    as many steps as the base mesh."""
    ratios = [Fraction(n, base) ** 2 for n in meshes]
    outer = 1
    for r in ratios:
        outer = outer * r.denominator // math.gcd(outer, r.denominator)
    return [int(r * outer) for r in ratios]


def coexistence(T_ratio):
    Tc = ppl.tc(EOS["a"], EOS["b"], EOS["R"])
    rv, rl, _ = ppl.maxwell(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], T_ratio * Tc)
    return Tc, rv, rl


def _refined(base_cfg, n_base, n, T_ratio):
    c = ppl.refine(base_cfg, n_base, n, T_ratio)
    return c, ppl.tc(c["a"], c["b"], c["R"])


def _angle(rho, mid):
    # 0 for a liquid film over the whole bottom wall (no base to read), else NaN if no cap
    try:
        return ppl.contact_angle(rho, 2, mid)
    except ppl.PplError:
        return 0.0 if float(np.min(rho[0, :])) > mid else float("nan")


def _batch(sims, subs, autotune_steps):
    """The sequence as one batch. Gravity-free FP32 meshes whose flow is periodic in x run the
    two-column kernel, so that the batch takes the persistent launch (its tiles overlap as a
    wavefront, faster than graph branches); the rows per tile are autotuned for it."""
    persistent = all(s.cfg.get("precision") == "fp32" and s.cfg["gx"] == 0.0 and s.cfg["gy"] == 0.0
                     and s.cfg["hydro_bc"][0] == W.PERIODIC and s.nx % 2 == 0 for s in sims)
    shapes = []
    for s in sims:
        if persistent:
            s.select_kernel("pair")
        shapes.append(s.autotune(autotune_steps)[0] if autotune_steps else s.launch()[0])
        if persistent and s.kernel != "pair":
            s.select_kernel("pair")
            shapes[-1] = s.launch()[0]
    return ppl.Batch(sims, subs), shapes


def droplet_vaporization_study(meshes=(128, 256, 512), R0=20.0, T_ratio=0.8, Tv_ratio=0.9, lam=0.25,
                               kappa=0.3, iso_steps=10000, coarse_steps=200000, sample_every=None,
                               width=3.0, precision="fp32", autotune_steps=64):
    """Sec. 4.1: a droplet (radius R0 on the first mesh) in vapour held at Tv on the boundary
    ring. Returns R(t) per mesh in first-mesh lengths, sampled every outer step, Eq.
    (relative-change-R) between successive meshes, and the slope of R^2(t) over the
    evaporation phase (the D^2 law)."""
    base_n = meshes[0]
    Tc, rv, rl = coexistence(T_ratio)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio * Tc)
    base, _ = W.droplet_vaporization(Tc, rv, rl, sigma, nx=base_n, ny=base_n, R0=R0, width=width,
                                     T_ratio=T_ratio, Tv_ratio=Tv_ratio, kappa=kappa, iso_steps=iso_steps,
                                     lam=lam, precision=precision)
    subs = substeps(meshes, base_n)
    if sample_every is not None and sample_every % subs[0]:
        raise ValueError("sample_every must be a multiple of %d coarse steps" % subs[0])
    sims, params = [], []
    for n in meshes:
        r = n / base_n
        c, Tcn = _refined(base, base_n, n, T_ratio)
        _, ic = W.droplet_vaporization(Tcn, rv, rl, c["sigma"], nx=n, ny=n, R0=R0 * r, width=width * r,
                                       T_ratio=T_ratio, Tv_ratio=Tv_ratio, kappa=c["kappa"],
                                       iso_steps=c["iso_steps"], lam=lam, precision=precision)
        sims.append(ppl.Simulation(c, *ic))
        params.append({"n": n, "a": c["a"], "sigma": c["sigma"], "kappa": c["kappa"], "iso_steps": c["iso_steps"]})
    batch, shapes = _batch(sims, subs, autotune_steps)
    per_outer = subs[0]
    every = max(1, (sample_every or per_outer) // per_outer)
    mid, band = 0.5 * (rv + rl), 0.05 * (rl - rv)
    R = [[] for _ in meshes]
    t = []
    t0 = time.perf_counter()
    outer = (coarse_steps // per_outer) // every * every
    for k in range(every, outer + 1, every):  # whole sampling intervals per call: graph replays
        batch.step(every)
        t.append(k * per_outer)
        for i, (s, n) in enumerate(zip(sims, meshes)):
            R[i].append(math.sqrt(s.phase_area(mid - band, mid + band) / math.pi) * base_n / n)
    wall = time.perf_counter() - t0
    nodes = sum(n * n * s for n, s in zip(meshes, subs)) * outer
    batch.close()
    for s in sims:
        s.close()
    dR = [ppl.relative_change(R[i], R[i + 1]) for i in range(len(meshes) - 1)]
    slopes = []
    tt = np.asarray(t, dtype=np.float64)
    for r in R:
        r2 = np.asarray(r) ** 2
        # evaporation phase: after the isothermal start, while the droplet keeps a quarter of
        # its initial area
        sel = (tt > iso_steps) & (r2 > 0.25 * R0 * R0)
        slopes.append(float(np.polyfit(tt[sel], r2[sel], 1)[0]) if sel.sum() >= 3 else float("nan"))
    return {"meshes": list(meshes), "substeps": subs, "launch_rows": shapes, "params": params, "t": t, "R": R,
            "delta_R": dR, "orders": [math.log(dR[i] / dR[i + 1]) / math.log(meshes[i + 1] / meshes[i])
                                      for i in range(len(dR) - 1)],
            "d2_slope": slopes, "seconds": wall, "mlups": nodes / wall / 1e6}


def contact_angle_study(meshes=(160, 240, 360, 540), model=W.CONTACT_PSI, value=4.0, coarse_steps=20000,
                        R0_frac=0.2, T_ratio=0.86, precision="fp32", autotune_steps=64):
    """Sec. 4.3.1: an isothermal droplet on the bottom wall relaxing to its static shape on
    every mesh. Returns the contact angle per mesh and the relative change of the density
    fields between successive meshes (Eqs. rel-diff-timestep at the final time, the
    Delta* rho of the paper's contact-angle table). value: rho_w (psi-based) or G_w."""
    base_n = meshes[0]
    Tc, rv, rl = coexistence(T_ratio)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio * Tc)
    kw = dict(contact_model=model, rho_w=value if model == W.CONTACT_PSI else 4.0,
              G_w=value if model == W.CONTACT_MOD_PSI else 0.0, precision=precision)
    base, _ = W.sessile_droplet(Tc, rv, rl, sigma, nx=base_n, ny=base_n, R0=R0_frac * base_n, **kw)
    subs = substeps(meshes, base_n)
    sims = []
    for n in meshes:
        r = n / base_n
        c, Tcn = _refined(base, base_n, n, T_ratio)
        _, ic = W.sessile_droplet(Tcn, rv, rl, c["sigma"], nx=n, ny=n, R0=R0_frac * n, width=3.0 * r, **kw)
        sims.append(ppl.Simulation(c, *ic))
    batch, shapes = _batch(sims, subs, autotune_steps)
    t0 = time.perf_counter()
    batch.step(max(1, coarse_steps // subs[0]))
    wall = time.perf_counter() - t0
    mid = 0.5 * (rv + rl)
    theta = [_angle(s.fields()["rho"], mid) for s in sims]
    rel = []
    for i in range(len(meshes) - 1):
        num, den = ppl.cross_norm(sims[i], sims[i + 1], "rho")
        rel.append(num / den)
    batch.close()
    for s in sims:
        s.close()
    return {"meshes": list(meshes), "model": "psi" if model == W.CONTACT_PSI else "mod_psi", "value": value,
            "theta": theta, "delta_rho": rel, "launch_rows": shapes, "seconds": wall}


def _static_angle(n, G_w, base_n, coarse_steps, T_ratio, R0_frac, precision):
    Tc, rv, rl = coexistence(T_ratio)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio * Tc)
    base, _ = W.sessile_droplet(Tc, rv, rl, sigma, nx=base_n, ny=base_n, R0=R0_frac * base_n,
                                contact_model=W.CONTACT_MOD_PSI, G_w=G_w, precision=precision)
    c, Tcn = _refined(base, base_n, n, T_ratio)
    _, ic = W.sessile_droplet(Tcn, rv, rl, c["sigma"], nx=n, ny=n, R0=R0_frac * n, width=3.0 * n / base_n,
                              contact_model=W.CONTACT_MOD_PSI, G_w=G_w, precision=precision)
    with ppl.Simulation(c, *ic) as s:
        s.step(int(round(coarse_steps * (n / base_n) ** 2)))
        return _angle(s.fields()["rho"], 0.5 * (rv + rl))


def G_w_search(meshes=(160, 240, 360, 540), G_w0=-0.8, coarse_steps=20000, tol=0.5, max_iter=10,
               T_ratio=0.86, R0_frac=0.2, precision="fp32"):
    """Sec. 4.3.1, the paper's G_w table: the modified psi-based model does not keep its
    contact angle under refinement; find per mesh the G_w that restores the angle (degrees)
    of the first mesh at G_w0. The angle falls as G_w grows more negative (stronger
    adhesion): the search brackets the target by steps of 0.05 from the previous mesh's
    G_w, then refines by false position; each evaluation is a run to the static shape.
    Returns the target angle and (G_w, theta, evaluations) per mesh."""
    base_n = meshes[0]
    target = _static_angle(base_n, G_w0, base_n, coarse_steps, T_ratio, R0_frac, precision)
    out = [{"n": base_n, "G_w": G_w0, "theta": target, "evaluations": 1}]
    g_prev = G_w0
    for n in meshes[1:]:
        evals = []

        def f(g):
            th = _static_angle(n, g, base_n, coarse_steps, T_ratio, R0_frac, precision)
            evals.append((g, th))
            return th - target

        ga, fa = g_prev, f(g_prev)
        step = -0.05 if fa > 0 else 0.05
        gb, fb = ga + step, f(ga + step)
        while math.isfinite(fa + fb) and fa * fb > 0 and len(evals) < max_iter:
            ga, fa = gb, fb
            gb, fb = gb + step, f(gb + step)
        side = 0
        while math.isfinite(fa + fb) and fa * fb <= 0 and len(evals) < max_iter and min(abs(fa), abs(fb)) > tol:
            gc = gb - fb * (gb - ga) / (fb - fa) if fb != fa else 0.5 * (ga + gb)
            fc = f(gc)
            if not math.isfinite(fc):
                break
            if fc * fb < 0:
                ga, fa = gb, fb
                side = 0
            else:  # Illinois step: halve the kept end's value twice in a row
                fa = 0.5 * fa if side == 1 else fa
                side = 1
            gb, fb = gc, fc
        g_best, th_best = min(evals, key=lambda e: abs(e[1] - target) if math.isfinite(e[1]) else 1e9)
        out.append({"n": n, "G_w": g_best, "theta": th_best, "evaluations": len(evals),
                    "trace": [list(e) for e in evals]})
        g_prev = g_best
    return {"target_theta": target, "meshes": out}


def pool_boiling_study(meshes=(160, 240, 360, 540), rho_wh=3.44, Th_ratio=1.2, coarse_steps=40000,
                       sample_every=320, tau=5120, m=4800, shift_stride=160, precision="fp32",
                       autotune_steps=64):
    """Sec. 4.3.2 with the paper's settings (walls at T_sat = 0.86 T_c, heater of a fifth of
    the width at Th, rho_w 6.50 / rho_wh / 0.38, liquid below half height, g = -2.5e-5 on
    the first mesh). Returns d^N(t) of rho and T between successive meshes at the output
    times (temperature as T / T_c of each mesh), their global D^N, the bottom-wall heat
    flux Q(t) per mesh (in first-mesh units), and the time shift
    delta of each coarser mesh against the finest at tau (Eq. rel-diff-minimize, search
    window +-m, all in first-mesh steps)."""
    base_n = meshes[0]
    T_ratio = 0.86
    Tc, rv, rl = coexistence(T_ratio)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio * Tc)
    subs = substeps(meshes, base_n)
    if sample_every % subs[0] or tau % subs[0]:
        raise ValueError("sample_every and tau must be multiples of %d coarse steps" % subs[0])

    def build(n):
        proto, _ = W.paper_pool_boiling(Tc, rv, rl, sigma, n=base_n, rho_wh=rho_wh, Th_ratio=Th_ratio,
                                        precision=precision, per_node=False)
        c, Tcn = _refined(proto, base_n, n, T_ratio)
        cfg, ic = W.paper_pool_boiling(Tcn, rv, rl, c["sigma"], n=n, rho_wh=rho_wh, Th_ratio=Th_ratio,
                                       g=-c["gy"], precision=precision)
        cfg.update(a=c["a"], kappa=c["kappa"])
        return cfg, ic

    cases = [build(n) for n in meshes]
    sims = [ppl.Simulation(c, *ic) for c, ic in cases]
    batch, shapes = _batch(sims, subs, autotune_steps)
    every = sample_every // subs[0]
    terms = {f: [[] for _ in meshes[1:]] for f in ("rho", "T")}
    Q = [[] for _ in meshes]
    t = []
    t0 = time.perf_counter()
    for k in range(every, coarse_steps // subs[0] + 1, every):
        batch.step(every)
        t.append(k * subs[0])
        for i in range(len(meshes) - 1):
            for f in ("rho", "T"):
                terms[f][i].append(ppl.cross_norm(sims[i], sims[i + 1], f))
        for i, s in enumerate(sims):
            Q[i].append(s.wall_heat_flux(2))
    wall = time.perf_counter() - t0
    batch.close()
    for s in sims:
        s.close()
    d = {f: [[a / b for a, b in pairs] for pairs in terms[f]] for f in terms}
    D = {f: [sum(a for a, _ in pairs) / sum(b for _, b in pairs) for pairs in terms[f]] for f in terms}

    # time shifts against the finest mesh at tau
    cf, icf = cases[-1]
    shifts = []
    with ppl.Simulation(cf, *icf) as finest:
        finest.step(tau * subs[-1] // subs[0])
        for (c, ic), n, sub in zip(cases[:-1], meshes[:-1], subs[:-1]):
            scale = sub / subs[0]
            with ppl.Simulation(c, *ic) as s:
                s.step(int(round((tau - m) * scale)))
                delta, num = ppl.time_shift(s, finest, int(round(m * scale)), int(round(shift_stride * scale)))
                shifts.append({"n": n, "delta": delta / scale, "num": num})
    # Q in first-mesh units: T scales with dx^2 (Table 1) and the wall gradient with 1/dx
    Q = [[q * (n / base_n) ** 3 for q in series] for series, n in zip(Q, meshes)]
    return {"meshes": list(meshes), "substeps": subs, "launch_rows": shapes, "t": t, "d": d, "D": D, "Q": Q,
            "shifts": shifts, "seconds": wall, "rho_wh": rho_wh, "Th_ratio": Th_ratio}


def _front(sim, rho_mid):
    """Interface position of a strip (Sec. 4.2): where the y-mean density first rises
    through rho_mid, by linear interpolation, in nodes from the wall at x = 0."""
    prof = sim.fields()["rho"].mean(axis=0)
    i = int(np.argmax(prof > rho_mid))
    if i == 0:
        return float("nan")
    return float(i - 1 + (rho_mid - prof[i - 1]) / (prof[i] - prof[i - 1]))


def stefan_study(param_set=2, meshes=(160, 320, 640, 1280, 2560), coarse_steps=20000, sample_every=200,
                 precision="fp64", autotune_steps=64):
    """Sec. 4.2, Table 3: the one-dimensional boiling-like problem on meshes of L nodes along
    x (4 nodes across, y periodic), all run as one batch with dt ~ dx^2. Liquid at T_sat =
    0.86 T_c, the psi-based hydrophobic wall at x = 0 held at T_w = 0.9 T_c, outflow at the
    far end, a vapour layer of 10 / 160 of the length. param_set 1: c_v = 5 and both
    diffusivities 0.3 (Ja = 0.038); 2: c_v = 10, lambda_l = 15, lambda_v = 1 (Ja = 0.076).
    Returns the interface position s(t) per mesh in first-mesh nodes and the relative change
    of Eq. (relative-change-R) form between successive meshes, with observed orders.

    FP64 by default: with dt ~ dx^2 the per-step change of T and rho on the finest meshes
    (256 steps per coarse step at 2560) falls to tens of FP32 ulps of the stored deviations,
    and over millions of steps the rounding drift of the FP32 path moves the front."""
    base_n = meshes[0]
    T_ratio = 0.86
    Tc, rv, rl = coexistence(T_ratio)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], T_ratio * Tc)
    if param_set == 1:
        cv, lam_v, lam_l = 5.0, 0.3 * rv * 5.0, 0.3 * rl * 5.0
    else:
        cv, lam_v, lam_l = 10.0, 1.0, 15.0
    kw = dict(cv=cv, lambda_v=lam_v, lambda_l=lam_l, dT_ratio=0.04, T_ratio=T_ratio, precision=precision)
    n_vap = 10.0 / 160.0
    base, _ = W.stefan_strip(Tc, rv, rl, sigma, nx=base_n, ny=4, n_vapour=n_vap * base_n, **kw)
    subs = substeps(meshes, base_n)
    if sample_every % subs[0]:
        raise ValueError("sample_every must be a multiple of %d coarse steps" % subs[0])
    sims = []
    for n in meshes:
        r = n / base_n
        c, Tcn = _refined(base, base_n, n, T_ratio)
        c["ny"] = 4  # the problem is one-dimensional: refine along x only
        _, ic = W.stefan_strip(Tcn, rv, rl, c["sigma"], nx=n, ny=4, n_vapour=n_vap * n, width=2.0 * r, **kw)
        sims.append(ppl.Simulation(c, *ic))
    batch, shapes = _batch(sims, subs, autotune_steps)
    mid = 0.5 * (rv + rl)
    every = sample_every // subs[0]
    s_t, t = [[] for _ in meshes], []
    t0 = time.perf_counter()
    for k in range(every, coarse_steps // subs[0] + 1, every):
        batch.step(every)
        t.append(k * subs[0])
        for i, (sim, n) in enumerate(zip(sims, meshes)):
            s_t[i].append(_front(sim, mid) * base_n / n)
    wall = time.perf_counter() - t0
    batch.close()
    for sim in sims:
        sim.close()
    ds = [ppl.relative_change(s_t[i], s_t[i + 1]) for i in range(len(meshes) - 1)]
    orders = [math.log(ds[i] / ds[i + 1]) / math.log(meshes[i + 2] / meshes[i + 1]) for i in range(len(ds) - 1)]
    return {"param_set": param_set, "meshes": list(meshes), "substeps": subs, "launch_rows": shapes, "t": t,
            "s": s_t, "delta_s": ds, "orders": orders, "seconds": wall}


def fp32_error_study(steps_scale=1.0):
    """The FP32 path (FP32 arithmetic, f - w rho_ref and T - T_ref stored in FP32) against the
    FP64 path (which matches the FP64 oracle to 1e-10) on the synthetic cases shaped like the
    paper's: per field, the relative L1 difference sum|a - b| / sum|b| (the form of Eq.
    rel-diff-timestep) and the pointwise maximum relative difference of rho and T, the bulk
    (coexistence) densities, the droplet radius R(t) of Sec. 4.1 and the Stefan interface
    position of Sec. 4.2 (where the y-mean density crosses rho_mid)."""
    out = {}
    Tc = ppl.tc(EOS["a"], EOS["b"], EOS["R"])

    def pair(cfg, ic, steps, probe=None, every=None):
        res = {}
        for prec in ("fp64", "fp32"):
            with ppl.Simulation(dict(cfg, precision=prec), *ic) as s:
                series = []
                done = 0
                while done < steps:
                    k = min(every or steps, steps - done)
                    s.step(k)
                    done += k
                    if probe:
                        series.append(probe(s))
                res[prec] = (s.fields(), series)
        return res

    def compare(res, extra=None):
        a, b = res["fp32"][0], res["fp64"][0]
        r = {}
        for f in ("rho", "T"):
            r[f + "_l1rel"] = float(np.abs(a[f] - b[f]).sum() / np.abs(b[f]).sum())
            r[f + "_maxrel"] = float(np.max(np.abs(a[f] - b[f]) / np.abs(b[f])))
        r["rho_min_rel"] = float(abs(a["rho"].min() - b["rho"].min()) / b["rho"].min())
        r["rho_max_rel"] = float(abs(a["rho"].max() - b["rho"].max()) / b["rho"].max())
        # pointwise in the bulk phases: nodes 8 or more nodes from every interface node
        rho = b["rho"]
        gap = float(rho.max() - rho.min())
        near = (rho > rho.min() + 0.1 * gap) & (rho < rho.max() - 0.1 * gap)
        for ax in (0, 1):
            grown = near.copy()
            for k in range(1, 9):
                grown |= np.roll(near, k, axis=ax) | np.roll(near, -k, axis=ax)
            near = grown
        e = np.abs(a["rho"] - rho) / rho
        r["rho_bulk_maxrel"] = float(e[~near].max()) if (~near).any() else float("nan")
        if extra:
            r.update(extra(res))
        return r

    n = lambda x: max(1, int(round(x * steps_scale)))
    # static droplet (64^2, 0.8 T_c, 5,000 steps)
    _, rv, rl = coexistence(0.8)
    cfg, ic = W.static_droplet(Tc, rv, rl, nx=64, ny=64, R0=16.0)
    out["static_droplet_64"] = compare(pair(cfg, ic, n(5000)))
    # Stefan strip (1024 x 4, 0.86 T_c + 0.05 T_c wall), interface position
    Tc_, rv, rl = coexistence(0.86)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], 0.86 * Tc)
    cfg, ic = W.stefan_strip(Tc, rv, rl, sigma, nx=1024, ny=4, n_vapour=10)
    mid = 0.5 * (rv + rl)

    def front(s):
        prof = s.fields()["rho"].mean(axis=0)
        i = int(np.argmax(prof > mid))
        return float(i - 1 + (mid - prof[i - 1]) / (prof[i] - prof[i - 1])) if i > 0 else float("nan")

    def front_err(res):
        a, b = np.array(res["fp32"][1]), np.array(res["fp64"][1])
        return {"front_max_abs_nodes": float(np.nanmax(np.abs(a - b))), "front_final": float(b[-1])}

    out["stefan_1024x4"] = compare(pair(cfg, ic, n(20000), front, n(2000)), front_err)
    # droplet vaporization (256^2, 0.8 / 0.9 T_c, kappa 0.3), radius R(t)
    _, rv, rl = coexistence(0.8)
    cfg, ic = W.droplet_vaporization(Tc, rv, rl, ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"],
                                                             0.8 * Tc), nx=256, ny=256, R0=40.0, iso_steps=n(2000))
    midv, band = 0.5 * (rv + rl), 0.05 * (rl - rv)
    radius = lambda s: math.sqrt(s.phase_area(midv - band, midv + band) / math.pi)

    def radius_err(res):
        a, b = np.array(res["fp32"][1]), np.array(res["fp64"][1])
        return {"radius_max_rel": float(np.max(np.abs(a - b) / b)), "radius_final": float(b[-1])}

    out["droplet_vaporization_256"] = compare(pair(cfg, ic, n(20000), radius, n(1000)), radius_err)
    # pool boiling (1024 x 2048): the vapour area over the heater (where the bubbles form) and
    # the pool's free-surface height as the interface measures
    _, rv, rl = coexistence(0.86)
    cfg, ic = W.pool_boiling(Tc, rv, rl, sigma, nx=1024, ny=2048)
    midp, bandp = 0.5 * (rv + rl), 0.05 * (rl - rv)

    def pool_measures(s):
        rho = s.fields()["rho"]
        frac = np.clip((rho - (midp - bandp)) / (2 * bandp), 0.0, 1.0)
        nx = rho.shape[1]
        heater = slice((nx - nx // 5) // 2, (nx + nx // 5) // 2)
        vapour_heater = float((1.0 - frac[: rho.shape[0] // 3, heater]).sum())
        col = frac.mean(axis=1)  # liquid fraction per row: the surface is where it falls through 1/2
        i = int(np.argmax(col < 0.5))
        surface = float(i - 1 + (col[i - 1] - 0.5) / (col[i - 1] - col[i])) if i > 0 else float("nan")
        return vapour_heater, surface

    def pool_err(res):
        a, b = res["fp32"][1][-1], res["fp64"][1][-1]
        return {"vapour_area_over_heater_rel": abs(a[0] - b[0]) / max(b[0], 1e-300),
                "vapour_area_over_heater": b[0], "surface_height_abs_nodes": abs(a[1] - b[1]),
                "surface_height": b[1]}

    out["pool_boiling_1024x2048"] = compare(pair(cfg, ic, n(2000), pool_measures, n(2000)), pool_err)
    return out


def batch_throughput(meshes=(128, 256, 512), outer=200, precision="fp32", autotune_steps=64):
    """The batched refinement sequence against stepping the same handles one after another:
    wall time of `outer` outer steps (1 : 4 : 16 steps per coarse step for 128^2 / 256^2 /
    512^2) each way, from the same initial states; the batch both as concurrent graph
    branches and as one persistent launch (FP32 two-column handles)."""
    base_n = meshes[0]
    Tc, rv, rl = coexistence(0.8)
    sigma = ppl.sigma_for(EOS["a"], EOS["b"], EOS["R"], EOS["omega"], EOS["G"], 0.8 * Tc)
    base, _ = W.droplet_vaporization(Tc, rv, rl, sigma, nx=base_n, ny=base_n, R0=base_n * 0.15,
                                     iso_steps=10 * outer, precision=precision)
    subs = substeps(meshes, base_n)

    def make():
        sims = []
        for n in meshes:
            c, Tcn = _refined(base, base_n, n, 0.8)
            _, ic = W.droplet_vaporization(Tcn, rv, rl, c["sigma"], nx=n, ny=n, R0=n * 0.15, width=3.0 * n / base_n,
                                           iso_steps=c["iso_steps"], precision=precision)
            s = ppl.Simulation(c, *ic)
            if autotune_steps:
                s.autotune(autotune_steps)
                if mode == "persistent" and s.kernel != "pair":
                    s.select_kernel("pair")  # the persistent launch runs the two-column kernel
            sims.append(s)
        return sims

    mode = "graph"
    sims = make()
    for s, k in zip(sims, subs):  # warm-up (graph capture)
        s.step(2 * k)
    t0 = time.perf_counter()
    for s, k in zip(sims, subs):
        s.step(outer * k)
    seq = time.perf_counter() - t0
    for s in sims:
        s.close()
    times = {}
    for mode in ("graph", "persistent") if precision == "fp32" else ("graph",):
        sims = make()
        with ppl.Batch(sims, subs, mode=mode) as b:
            b.step(2)
            if mode == "persistent":
                b.step(outer)  # capture of the launch for this outer count
            t0 = time.perf_counter()
            b.step(outer)
            times[mode] = time.perf_counter() - t0
        for s in sims:
            s.close()
    bat = times["graph"]
    nodes = sum(n * n * k for n, k in zip(meshes, subs)) * outer
    out = {"meshes": list(meshes), "substeps": subs, "outer": outer, "sequential_s": seq, "batch_s": bat,
           "speedup": seq / bat, "batch_mlups": nodes / bat / 1e6, "sequential_mlups": nodes / seq / 1e6}
    if "persistent" in times:
        out.update(persistent_s=times["persistent"], persistent_mlups=nodes / times["persistent"] / 1e6)
    return out
