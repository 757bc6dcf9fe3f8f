"""GPU: the mesh-refinement tools of the library through the C ABI — the cross-mesh
difference (Eqs. rel-diff-timestep, global-rel-diff) against the oracle's on oracle-run
fields, the batched refinement sequence (Sec. 3: dt ~ dx^2 substeps) against separately
stepped handles, and the launch-shape setter / autotuner (results unchanged)."""
import numpy as np
import pytest

import workloads as W
from oracle import norms, oracle, thermo

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


def droplet(th, n, precision="fp64", **kw):
    e = th["e"]
    rv, rl, _ = th[0.8]
    return W.static_droplet(e.Tc, rv, rl, nx=n, ny=n, R0=n / 4.0, width=3.0 * n / 40, precision=precision, **kw)


def pool(th, nx, ny):
    e = th["e"]
    rv, rl, _ = th[0.86]
    return W.pool_boiling(e.Tc, rv, rl, 0.1032, nx=nx, ny=ny, g=3e-5)


@pytest.mark.parametrize("case", ["droplet", "pool"])
def test_cross_norm_matches_oracle(ppl, th, case):
    # two meshes of one problem, each advanced on the GPU and in the oracle; the GPU
    # difference of the GPU fields against the oracle difference of the oracle fields
    if case == "droplet":
        (cc, icc), (cf, icf), steps, px, py = droplet(th, 40), droplet(th, 61), (30, 60), True, True
    else:
        (cc, icc), (cf, icf), steps, px, py = pool(th, 48, 40), pool(th, 73, 61), (40, 90), True, False
    sc, sf = ppl.Simulation(cc, *icc), ppl.Simulation(cf, *icf)
    sc.step(steps[0])
    sf.step(steps[1])
    oc, of = oracle.Oracle(cc, *icc), oracle.Oracle(cf, *icf)
    oc.step(steps[0])
    of.step(steps[1])
    foc, fof = oc.fields(), of.fields()
    # temperatures compare as T / T_c of each mesh
    foc["T"], fof["T"] = foc["T"] / oracle.tc(cc), fof["T"] / oracle.tc(cf)
    for field in ("rho", "T"):
        num, den = ppl.cross_norm(sc, sf, field)
        wnum, wden = norms.rel_diff_terms(foc[field], fof[field], px, py)
        # the two states agree to the FP64 parity bound (1e-10 relative)
        assert den == pytest.approx(wden, rel=1e-10)
        assert num == pytest.approx(wnum, rel=1e-8, abs=1e-10 * wden)
    # same handle against itself: zero difference
    num, den = ppl.cross_norm(sf, sf, "rho")
    assert num < 1e-14 * den
    sc.close()
    sf.close()


def test_cross_norm_rejects_different_boundaries(ppl, th):
    (c1, i1), (c2, i2) = droplet(th, 40), pool(th, 48, 40)
    a, b = ppl.Simulation(c1, *i1), ppl.Simulation(c2, *i2)
    with pytest.raises(ppl.PplError):
        ppl.cross_norm(a, b, "rho")
    a.close()
    b.close()


def _sequence(ppl, th, precision):
    base, ic = droplet(th, 24, precision=precision, kappa=0.2)
    base.update(gy=-2e-5, energy_on=1, iso_steps=5, cv=6.0, lambda_l=0.2, lambda_v=0.2)
    cfgs, ics = [], []
    for n in (24, 48, 96):
        c = ppl.refine(base, 24, n, 0.8)
        c.update(precision=precision)
        cfgs.append(c)
        _, icn = droplet(th, n, precision=precision)
        rho, ux, uy, _ = icn
        ics.append((rho, ux, uy, np.full_like(rho, c["T_ref"])))
    return cfgs, ics


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("subs,outer", [((1, 4, 16), 3), ((1, 2, 3), 7)])
def test_batch_equals_separate_handles(ppl, th, precision, subs, outer):
    cfgs, ics = _sequence(ppl, th, precision)
    batch_sims = [ppl.Simulation(c, *ic) for c, ic in zip(cfgs, ics)]
    with ppl.Batch(batch_sims, subs) as b:
        b.step(outer)
        b.step(1)
    for k, (c, ic) in enumerate(zip(cfgs, ics)):
        ref = ppl.Simulation(c, *ic)
        ref.step((outer + 1) * subs[k])
        np.testing.assert_array_equal(batch_sims[k].populations(), ref.populations())
        np.testing.assert_array_equal(batch_sims[k].fields()["T"], ref.fields()["T"])
        assert batch_sims[k].launch_count == ref.launch_count == (outer + 1) * subs[k]
        ref.close()
        # the handle keeps stepping on its own after the batch
        batch_sims[k].step(3)
        batch_sims[k].close()


def test_batch_rejects_bad_arguments(ppl, th):
    c, ic = droplet(th, 24)
    s = ppl.Simulation(c, *ic)
    with pytest.raises(ppl.PplError):
        ppl.Batch([s, s], [1, 4])  # the same handle twice
    with pytest.raises(ppl.PplError):
        ppl.Batch([s], [0])
    s.close()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_launch_shape_does_not_change_results(ppl, th, precision, rtol):
    # gravity off: the domain-mass sum (the only shape-dependent rounding) does not enter;
    # interior and boundary row blocks are separate compiled specialisations, so only
    # contraction-level rounding may differ
    c, ic = droplet(th, 70, precision=precision, kappa=0.3)
    c["nx"] = c["ny"] = 70
    ref = ppl.Simulation(c, *ic)
    ref.step(40)
    want = ref.populations()
    ref.close()
    for rows in (1, 3, 8, 13, 70):
        s = ppl.Simulation(c, *ic)
        s.set_launch(rows)
        assert s.launch()[0] == rows
        s.step(40)
        np.testing.assert_allclose(s.populations(), want, rtol=rtol, atol=rtol * 1e-2)
        s.close()


@pytest.mark.parametrize("g", [0.0, 3e-5])
def test_two_height_launch_shape(ppl, th, g):
    # a grid large enough for the default two-column shape to follow one wave of tall row
    # blocks with short ones (pool boiling, 2048 x 1800): results agree with one uniform wave
    # to contraction-level rounding (with gravity, the per-CTA mass partials also round
    # differently in the domain-mean density)
    e = th["e"]
    rv, rl, _ = th[0.86]
    c, ic = W.pool_boiling(e.Tc, rv, rl, 0.1032, nx=2048, ny=1800, g=g, precision="fp32")
    s = ppl.Simulation(c, *ic)
    assert s.kernel == "pair"
    rows, ctas = s.launch()
    strips = -(-2048 // 120)
    assert ctas > strips * -(-1800 // rows)  # short row blocks follow the tall ones
    s.step(30)
    got = s.fields()
    assert s.norms()["flags"] == 0
    s.set_launch(rows)  # uniform blocks of the tall height
    assert s.launch() == (rows, strips * -(-1800 // rows))
    s.close()
    ref = ppl.Simulation(c, *ic)
    ref.set_launch(rows)
    ref.step(30)
    want = ref.fields()
    ref.close()
    for k in ("rho", "T"):
        np.testing.assert_allclose(got[k], want[k], rtol=1e-5, atol=1e-7)


def test_autotune_restores_state(ppl, th):
    c, ic = pool(th, 300, 160)
    c.update(gy=-3e-5)
    s = ppl.Simulation(c, *ic)
    s.step(10)
    f0, n0 = s.populations(), s.launch_count
    rows, ms = s.autotune(8)
    assert rows >= 1 and ms > 0
    assert s.launch()[0] == rows
    np.testing.assert_array_equal(s.populations(), f0)
    assert s.launch_count == n0
    s.step(50)
    got = s.fields()
    s.set_launch(0)
    s.close()
    ref = ppl.Simulation(c, *ic)
    ref.step(60)
    want = ref.fields()
    ref.close()
    # gravity on: the per-CTA mass partials round differently, nothing else differs
    for k in ("rho", "T"):
        np.testing.assert_allclose(got[k], want[k], rtol=1e-12)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_phase_area_matches_oracle(ppl, th, precision, rtol):
    e = th["e"]
    rv, rl, _ = th[0.8]
    cfg, ic = W.droplet_vaporization(e.Tc, rv, rl, 0.1, nx=60, ny=52, R0=12.0, iso_steps=40, precision=precision)
    s = ppl.Simulation(cfg, *ic)
    s.step(160)
    o = oracle.Oracle(cfg, *ic)
    o.step(160)
    rho = o.fields()["rho"]
    for lo, hi in ((rv, rl), (0.5 * (rv + rl) - 0.1, 0.5 * (rv + rl) + 0.1)):
        assert s.phase_area(lo, hi) == pytest.approx(norms.phase_area(rho, lo, hi), rel=rtol)
    with pytest.raises(ppl.PplError):
        s.phase_area(rl, rv)
    s.close()


def test_time_shift_search(ppl, th):
    # Eq. (rel-diff-minimize): the same mesh as "finest" has its minimum, exactly zero, at
    # delta = 0; a finer mesh's minimum and its value agree with the oracle's scan
    (cc, icc), (cf, icf) = droplet(th, 40, kappa=0.2), droplet(th, 61, kappa=0.2)
    tau, m, stride = 60, 30, 10
    fine = ppl.Simulation(cc, *icc)
    fine.step(tau)
    c = ppl.Simulation(cc, *icc)
    c.step(tau - m)
    d, num = ppl.time_shift(c, fine, m, stride)
    assert (d, num) == (0, 0.0)
    c.close()
    fine.close()

    fine = ppl.Simulation(cf, *icf)
    fine.step(tau)
    c = ppl.Simulation(cc, *icc)
    c.step(tau - m)
    d, num = ppl.time_shift(c, fine, m, stride)
    of = oracle.Oracle(cf, *icf)
    of.step(tau)
    ff = of.fields()["rho"]
    oc = oracle.Oracle(cc, *icc)
    oc.step(tau - m)
    scan = []
    for k, shift in enumerate(range(-m, m + 1, stride)):
        if k:
            oc.step(stride)
        scan.append((norms.rel_diff_terms(oc.fields()["rho"], ff, True, True)[0], shift))
    wnum, wd = min(scan)
    assert d == wd
    assert num == pytest.approx(wnum, rel=1e-8)
    c.close()
    fine.close()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("fp32", 2e-3)])
def test_wall_heat_flux_matches_oracle(ppl, th, precision, rtol):
    # Eq. (pool-heat-flux) through the heated bottom wall and the adiabatic top wall
    e = th["e"]
    rv, rl, _ = th[0.86]
    cfg, ic = W.pool_boiling(e.Tc, rv, rl, 0.1032, nx=64, ny=48, g=3e-5, precision=precision)
    s = ppl.Simulation(cfg, *ic)
    s.step(120)
    o = oracle.Oracle(cfg, *ic)
    o.step(120)
    fo = o.fields()
    for side in (2, 3):
        want = norms.wall_heat_flux(fo["rho"], fo["T"], side, cfg["rho_v"], cfg["rho_l"], cfg["lambda_v"],
                                    cfg["lambda_l"])
        scale = abs(norms.wall_heat_flux(fo["rho"], fo["T"], 2, cfg["rho_v"], cfg["rho_l"], cfg["lambda_v"],
                                         cfg["lambda_l"]))
        assert s.wall_heat_flux(side) == pytest.approx(want, rel=rtol, abs=rtol * scale)
    assert s.wall_heat_flux(2) > 0  # the heater feeds heat into the pool
    with pytest.raises(ppl.PplError):
        s.wall_heat_flux(0)  # periodic side
    s.close()


def _sequence_fp32(ppl, th, ns, g=-2e-5):
    base, _ = droplet(th, ns[0], precision="fp32", kappa=0.2)
    base.update(gy=g, energy_on=1, iso_steps=5, cv=6.0, lambda_l=0.2, lambda_v=0.2)
    cfgs, ics = [], []
    for n in ns:
        c = ppl.refine(base, ns[0], n, 0.8)
        c.update(precision="fp32")
        cfgs.append(c)
        _, icn = droplet(th, n, precision="fp32")
        rho, ux, uy, _ = icn
        ics.append((rho, ux, uy, np.full_like(rho, c["T_ref"])))
    return cfgs, ics


@pytest.mark.parametrize("ns,subs,outer,g", [((24, 48, 96), (1, 4, 16), 3, -2e-5), ((64, 128, 256), (1, 4, 16), 2, -2e-5),
                                             ((32, 48, 64), (1, 2, 3), 5, -2e-5), ((24, 48, 96), (1, 4, 16), 3, 0.0),
                                             ((64, 128, 256), (1, 4, 16), 2, 0.0), ((32, 48, 64), (1, 2, 3), 5, 0.0)])
def test_persistent_batch_equals_separate_handles(ppl, th, ns, subs, outer, g):
    # one persistent launch per call over every mesh's steps (with gravity each step waits for
    # its mesh's domain-mean density; without, a tile waits for the tiles within its reach,
    # a wavefront; the energy equation switches on during the run); the separately stepped
    # 256^2 handle stages rows by TMA, the batch by per-thread copies
    cfgs, ics = _sequence_fp32(ppl, th, ns, g)
    sims = [ppl.Simulation(c, *ic) for c, ic in zip(cfgs, ics)]
    with ppl.Batch(sims, subs, mode="persistent") as b:
        assert b.mode == "persistent"
        b.step(outer)
        b.step(1)
    for k, (c, ic) in enumerate(zip(cfgs, ics)):
        ref = ppl.Simulation(c, *ic)
        ref.step((outer + 1) * subs[k])
        np.testing.assert_array_equal(sims[k].populations(), ref.populations())
        np.testing.assert_array_equal(sims[k].fields()["T"], ref.fields()["T"])
        assert sims[k].norms()["mass"] == ref.norms()["mass"]
        assert sims[k].launch_count == ref.launch_count == (outer + 1) * subs[k]
        ref.close()
        sims[k].step(3)  # the handle keeps stepping on its own
        sims[k].close()


def test_persistent_batch_dirichlet_ring(ppl, th):
    # droplets in superheated vapour held by a Dirichlet temperature ring: every strip of these
    # small meshes holds a Dirichlet x line, so the persistent kernel runs its tiles with rows
    # inside the domain in the form that keeps only the per-column Dirichlet checks (the step
    # kernel runs them in its general form); the energy equation switches on during the run
    e = th["e"]
    rv, rl, _ = th[0.8]
    cfgs, ics = [], []
    for n in (64, 128, 256):
        c, ic = W.droplet_vaporization(e.Tc, rv, rl, thermo.sigma_for(e, 0.8 * e.Tc), nx=n, ny=n, R0=n / 4.0,
                                       iso_steps=4, precision="fp32")
        cfgs.append(c)
        ics.append(ic)
    subs = (1, 4, 16)
    sims = [ppl.Simulation(c, *ic) for c, ic in zip(cfgs, ics)]
    with ppl.Batch(sims, subs, mode="persistent") as b:
        assert b.mode == "persistent"
        b.step(3)
    for k, (c, ic) in enumerate(zip(cfgs, ics)):
        ref = ppl.Simulation(c, *ic)
        ref.step(3 * subs[k])
        np.testing.assert_array_equal(sims[k].populations(), ref.populations())
        np.testing.assert_array_equal(sims[k].fields()["T"], ref.fields()["T"])
        assert sims[k].norms()["flags"] == 0
        ref.close()
        sims[k].close()


def test_persistent_batch_wait_limit_runs_out(ppl, th):
    # a zero wait limit makes the first dependency wait give up: the launch stops, the call
    # reports PPL_E_TIMEOUT, nothing faults, and the handles step normally after a reset
    cfgs, ics = _sequence_fp32(ppl, th, (64, 128, 256))
    sims = [ppl.Simulation(c, *ic) for c, ic in zip(cfgs, ics)]
    b = ppl.Batch(sims, (1, 4, 16), mode="persistent")
    b.set_wait_limit(0)
    with pytest.raises(ppl.PplError) as err:
        b.step(2)
    assert err.value.code == ppl.PPL_E_TIMEOUT
    b.set_wait_limit(1_000_000_000)
    for s, ic in zip(sims, ics):
        s.reset(*ic)
    b.step(1)
    for s in sims:
        assert s.norms()["flags"] == 0
    b.close()
    for s in sims:
        s.close()


def test_persistent_batch_needs_two_column_fp32_handles(ppl, th):
    c, ic = droplet(th, 24)  # FP64
    s = ppl.Simulation(c, *ic)
    b = ppl.Batch([s], [1])
    with pytest.raises(ppl.PplError):
        b.set_mode("persistent")
    assert b.mode == "auto"  # the default, which runs graphs for this handle
    b.close()
    s.close()
