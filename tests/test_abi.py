"""The C-ABI library loads and exports every entry point declared in include/ppl.h;
its host-side helpers agree with the oracle's thermodynamics (no GPU needed)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ppl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ppl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_04560_gb300 import ppl
    return ppl.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    raw = ctypes.CDLL(lib._name)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_strerror_names_every_code(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.ppl_strerror(code) not in (None, b"", b"unknown error code")
    assert lib.ppl_strerror(-99) == b"unknown error code"


def test_host_helpers_match_oracle_thermo():
    from oracle import thermo
    from paper_2201_04560_gb300 import ppl
    e = thermo.PR()
    assert ppl.tc(e.a, e.b, e.R) == e.Tc
    for tr in (0.6, 0.8, 0.86, 0.95):
        rv, rl, ps = ppl.maxwell(e.a, e.b, e.R, e.omega, tr * e.Tc)
        ov, ol, ops = thermo.maxwell(e, tr * e.Tc)
        assert rv == pytest.approx(ov, rel=1e-9)
        assert rl == pytest.approx(ol, rel=1e-9)
        assert ps == pytest.approx(ops, rel=1e-9)
    assert ppl.refine_a(3 / 49, 128, 192) == pytest.approx(thermo.refine_a(3 / 49, 128, 192), rel=1e-15)


def test_invalid_arguments_rejected_without_gpu(lib):
    rv, rl, ps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    from paper_2201_04560_gb300 import ppl
    # T above T_c has no coexistence
    assert lib.ppl_maxwell(3 / 49, 2 / 21, 1.0, 0.344, 1.0, ctypes.byref(rv), ctypes.byref(rl),
                           ctypes.byref(ps)) == ppl.PPL_E_INVAL
    h = ctypes.c_void_p()
    assert lib.ppl_init(None, None, None, None, None, ctypes.byref(h)) == ppl.PPL_E_INVAL
    # the wait-limit probe checks its limit (1 ns .. 1 s) and output before touching the device
    flags = ctypes.c_uint32(0)
    assert lib.ppl_stall_probe(0, ctypes.byref(flags)) == ppl.PPL_E_INVAL
    assert lib.ppl_stall_probe(2_000_000_000, ctypes.byref(flags)) == ppl.PPL_E_INVAL
    assert lib.ppl_stall_probe(1000, None) == ppl.PPL_E_INVAL
    assert lib.ppl_tma_staging(None) == ppl.PPL_E_INVAL
    # the FP64 rate probe checks its arguments before touching the device
    r = ctypes.c_double(0.0)
    assert lib.ppl_fp64_rate(0, ctypes.byref(r)) == ppl.PPL_E_INVAL
    assert lib.ppl_fp64_rate(10, None) == ppl.PPL_E_INVAL


def test_config_validation_rejects_bad_boundaries(lib):
    # validation runs before any CUDA call, so this needs no GPU
    import numpy as np

    import workloads as W
    from paper_2201_04560_gb300 import ppl
    z = np.zeros((8, 8))
    bad = [
        dict(hydro_bc=[W.WALL, W.PERIODIC, W.PERIODIC, W.PERIODIC]),           # half-periodic axis
        dict(hydro_bc=[W.WALL, W.WALL, W.WALL, W.WALL]),                       # wall corners
        dict(s=[1.0] * 8 + [2.5]),                                             # unstable rate
        dict(G=1.0),                                                           # psi needs G < 0
        dict(thermal_bc=[W.T_DIRICHLET, W.T_PERIODIC, W.T_PERIODIC, W.T_PERIODIC]),
    ]
    for kw in bad:
        cfg = W.base_config(8, 8, **kw)
        C, keep = ppl.make_config(cfg)
        h = ctypes.c_void_p()
        p = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        assert lib.ppl_init(ctypes.byref(C), p, p, p, p, ctypes.byref(h)) == ppl.PPL_E_INVAL, kw


def test_refinement_tools_match_oracle():
    # product-side sigma / gamma / kappa (Sec. 3.2) against the oracle's quadratures
    from oracle import thermo
    from paper_2201_04560_gb300 import ppl
    e = thermo.PR()
    for L in (128, 192, 288):
        a = thermo.refine_a(3 / 49, 128, L)
        el = thermo.PR(a=a)
        T = 0.86 * el.Tc
        assert ppl.sigma_for(a, el.b, el.R, el.omega, el.G, T) == pytest.approx(thermo.sigma_for(el, T), rel=1e-10)
    T = 0.8 * e.Tc
    for sig, kap in ((0.1, 0.0), (0.1032, 0.3)):
        g = ppl.gamma_planar(e.a, e.b, e.R, e.omega, e.G, T, sig, kap)
        assert g == pytest.approx(thermo.planar_gamma(e, T, sig, kap), rel=1e-7)
    e0 = thermo.PR()
    s0 = thermo.sigma_for(e0, 0.86 * e0.Tc)
    e1 = thermo.PR(a=thermo.refine_a(3 / 49, 128, 192))
    s1 = thermo.sigma_for(e1, 0.86 * e1.Tc)
    k = thermo.kappa_for(e0, e1, 0.86, 128, 192, s0, s1)
    assert ppl.kappa_for(3 / 49, 128, 192, e.b, e.R, e.omega, e.G, 0.86) == pytest.approx(k, abs=1e-7)


def test_refine_applies_table1_scaling():
    # Table 1 / Eq. (a-deltax): a ~ dx^2, T ~ dx^2 (with T_c), g ~ dx^3, grid ~ 1/dx
    import workloads as W
    from paper_2201_04560_gb300 import ppl
    Tc = ppl.tc(3 / 49, 2 / 21, 1.0)
    base = W.base_config(128, 64, gy=-2.5e-5, sigma=0.103, T_side=[0.9 * Tc] * 4, T_ref=0.86 * Tc,
                         hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                         thermal_bc=[W.T_PERIODIC, W.T_PERIODIC, W.T_DIRICHLET, W.T_DIRICHLET])
    out = ppl.refine(base, 128, 192, 0.86)
    r = 192 / 128
    assert (out["nx"], out["ny"]) == (192, 96)
    assert out["a"] == pytest.approx(3 / 49 / r ** 2, rel=1e-14)
    assert out["gy"] == pytest.approx(-2.5e-5 / r ** 3, rel=1e-14)
    assert out["T_side"][2] == pytest.approx(0.9 * Tc / r ** 2, rel=1e-12)
    base["iso_steps"] = 10000
    assert ppl.refine(base, 128, 192, 0.86)["iso_steps"] == 22500  # dt ~ dx^2
    assert out["sigma"] == pytest.approx(0.115, abs=5e-4)     # Table 2, L = 192
    assert 1 - out["kappa"] == pytest.approx(1 + 5.17e-2, rel=1e-2)  # Sec. 3.2


def test_relative_change_matches_oracle():
    # Eq. (relative-change-R), the library's host routine against the oracle's
    import numpy as np
    from oracle import norms
    from paper_2201_04560_gb300 import ppl
    rng = np.random.default_rng(2)
    R, Rs = 20 + rng.random(300), 20 + rng.random(300)
    assert ppl.relative_change(R, Rs) == pytest.approx(norms.relative_change_R(R, Rs), rel=1e-13)
    with pytest.raises(ppl.PplError):
        ppl.relative_change(R[:0], Rs[:0])
    with pytest.raises(ppl.PplError):
        ppl.relative_change(R[:3], np.zeros(3))


@pytest.mark.parametrize("side", [0, 1, 2, 3])
@pytest.mark.parametrize("yc", [-12.0, 0.0, 10.0])
def test_contact_angle_matches_oracle_on_caps(side, yc):
    # the library's host routine against the oracle's on a circular cap cut by a wall line,
    # for each of the four sides (the field is rotated so that the wall is that side)
    import numpy as np
    from oracle import norms
    from paper_2201_04560_gb300 import ppl
    nx, ny, R, W = 150, 80, 28.0, 3.0
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = 0.38 + 0.5 * (6.5 - 0.38) * (1 + np.tanh(2 * (R - np.hypot(x - 70.6, y - yc)) / W))
    mid = 0.5 * (6.5 + 0.38)
    want = norms.contact_angle(rho, mid)
    assert want == pytest.approx(90.0 + np.degrees(np.arcsin(yc / R)), abs=1.0)
    field = {2: rho, 3: rho[::-1, :], 0: rho.T, 1: rho.T[:, ::-1]}[side]
    assert ppl.contact_angle(field, side, mid) == pytest.approx(want, abs=1e-9)


def test_pressure_matches_oracle_eos():
    from oracle import thermo
    from paper_2201_04560_gb300 import ppl
    e = thermo.PR()
    for tr in (0.8, 0.86, 1.2):
        T = tr * e.Tc
        for rho in (0.3, 2.0, 6.5):
            p, dp = ppl.pressure(e.a, e.b, e.R, e.omega, T, rho)
            assert p == pytest.approx(float(e.p(rho, T)), rel=1e-13)
            h = 1e-5
            assert dp == pytest.approx((float(e.p(rho + h, T)) - float(e.p(rho - h, T))) / (2 * h), rel=1e-8)


@pytest.mark.parametrize("side", [0, 1, 2, 3])
def test_contact_angle_base_above_a_wall_layer_matches_oracle(side):
    import numpy as np
    from oracle import norms
    from paper_2201_04560_gb300 import ppl
    nx, ny, R, W, yc = 160, 90, 30.0, 3.0, -8.0
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = 0.38 + 0.5 * (6.5 - 0.38) * (1 + np.tanh(2 * (R - np.hypot(x - 80.3, y - yc)) / W))
    rho[0, :] = np.minimum(rho[0, :], 2.0)
    mid = 0.5 * (6.5 + 0.38)
    want = norms.contact_angle(rho, mid)
    field = {2: rho, 3: rho[::-1, :], 0: rho.T, 1: rho.T[:, ::-1]}[side]
    assert ppl.contact_angle(field, side, mid) == pytest.approx(want, abs=1e-9)
    film = np.where(y < 10, 6.5, 0.38)
    with pytest.raises(ppl.PplError):
        ppl.contact_angle({2: film, 3: film[::-1, :], 0: film.T, 1: film.T[:, ::-1]}[side], side, mid)
