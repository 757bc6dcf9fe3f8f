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
