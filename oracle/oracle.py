"""ctypes front end of the C FP64 oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use it. It builds its own shared object with gcc
(``-O2 -ffp-contract=off``, single-threaded) and shares nothing with the CUDA
library. The configuration is a plain dict (the schema of ``workloads``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PU8 = ctypes.POINTER(ctypes.c_uint8)


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("a", _D), ("b", _D), ("R", _D), ("omega", _D), ("G", _D),
        ("s", _D * 9),
        ("eta_l", _D), ("eta_v", _D), ("rho_l", _D), ("rho_v", _D),
        ("sigma", _D), ("kappa", _D), ("gx", _D), ("gy", _D), ("cv", _D),
        ("lambda_l", _D), ("lambda_v", _D),
        ("energy_on", ctypes.c_int32), ("iso_steps", ctypes.c_int64),
        ("hydro_bc", ctypes.c_int32 * 4), ("thermal_bc", ctypes.c_int32 * 4),
        ("T_side", _D * 4), ("rho_w_side", _D * 4),
        ("rho_w", _PD * 4), ("T_w", _PD * 4), ("T_dirichlet", _PU8 * 4),
        ("rho_bar_fixed", _D),
        ("contact_model", ctypes.c_int32), ("G_w", _D),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, plain -O2)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=c11", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_params_size.restype = ctypes.c_size_t
        assert L.orc_params_size() == ctypes.sizeof(OrcParams), "oracle struct layout mismatch"
        L.orc_init.argtypes = [ctypes.POINTER(OrcParams)] + [_PD] * 6
        L.orc_init.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.POINTER(OrcParams), _PD, _PD, ctypes.c_int64]
        L.orc_step.restype = ctypes.c_long
        L.orc_fields.argtypes = [ctypes.POINTER(OrcParams), _PD, _PD, _PD, _PD, _PD, _PD]
        L.orc_fields.restype = ctypes.c_long
        L.orc_energy_rhs.argtypes = [ctypes.POINTER(OrcParams)] + [_PD] * 5
        L.orc_energy_rhs.restype = ctypes.c_int
        L.orc_matrix.argtypes = [_PD, _PD]
        L.orc_tc.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_tc.restype = _D
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_PD)


def make_params(cfg: dict):
    """Marshal a config dict into the oracle struct; returns (struct, keepalive list)."""
    P = OrcParams()
    keep = []
    P.nx, P.ny = int(cfg["nx"]), int(cfg["ny"])
    for k in ("a", "b", "R", "omega", "G", "eta_l", "eta_v", "rho_l", "rho_v", "sigma", "kappa",
              "gx", "gy", "cv", "lambda_l", "lambda_v"):
        setattr(P, k, float(cfg[k]))
    for i in range(9):
        P.s[i] = float(cfg["s"][i])
    P.rho_bar_fixed = float(cfg.get("rho_bar_fixed", float("nan")))
    P.contact_model = int(cfg.get("contact_model", 0))
    P.G_w = float(cfg.get("G_w", 0.0))
    P.energy_on = int(cfg["energy_on"])
    P.iso_steps = int(cfg["iso_steps"])
    for sd in range(4):
        P.hydro_bc[sd] = int(cfg["hydro_bc"][sd])
        P.thermal_bc[sd] = int(cfg["thermal_bc"][sd])
        P.T_side[sd] = float(cfg["T_side"][sd])
        P.rho_w_side[sd] = float(cfg["rho_w_side"][sd])
        for name, dt, ptr in (("rho_w", np.float64, _PD), ("T_w", np.float64, _PD),
                              ("T_dirichlet", np.uint8, _PU8)):
            arr = (cfg.get(name) or [None] * 4)[sd]
            if arr is None:
                getattr(P, name)[sd] = ctypes.cast(None, ptr)
            else:
                a = np.ascontiguousarray(arr, dtype=dt)
                keep.append(a)
                getattr(P, name)[sd] = a.ctypes.data_as(ptr)
    return P, keep


class Oracle:
    """FP64 single-threaded reference simulation (state f[9][ny][nx], T[ny][nx])."""

    def __init__(self, cfg: dict, rho0, ux0, uy0, T0):
        self.cfg = dict(cfg)
        self.P, self._keep = make_params(cfg)
        ny, nx = int(cfg["ny"]), int(cfg["nx"])
        self.shape = (ny, nx)
        self.f = np.zeros((9, ny, nx), dtype=np.float64)
        self.T = np.zeros((ny, nx), dtype=np.float64)
        args = [np.ascontiguousarray(v, dtype=np.float64).reshape(ny, nx) for v in (rho0, ux0, uy0, T0)]
        lib().orc_init(ctypes.byref(self.P), *[_p(a) for a in args], _p(self.f), _p(self.T))
        self.step_count = 0

    def step(self, n: int = 1):
        for _ in range(int(n)):
            err = lib().orc_step(ctypes.byref(self.P), _p(self.f), _p(self.T), self.step_count)
            if err:
                raise FloatingPointError("oracle step failed (code %d) at step %d" % (err, self.step_count))
            self.step_count += 1

    def fields(self):
        ny, nx = self.shape
        rho = np.empty((ny, nx)); ux = np.empty((ny, nx)); uy = np.empty((ny, nx))
        rb = ctypes.c_double()
        err = lib().orc_fields(ctypes.byref(self.P), _p(self.f), _p(self.T), _p(rho), _p(ux), _p(uy),
                               ctypes.byref(rb))
        if err:
            raise FloatingPointError("oracle fields failed (code %d)" % err)
        return {"rho": rho, "ux": ux, "uy": uy, "T": self.T.copy(), "rho_bar": rb.value}


def window_step(cfg: dict, fields, x0: int, x1: int, y0: int, y1: int, rho_bar: float, steps: int = 1):
    """Advance a window [y0, y1) x [x0, x1) of a larger domain by `steps` steps.

    The window is padded by 3 * steps nodes on every side that is open (not a domain
    wall); padded columns/rows wrap around the periodic axes of the domain. The domain-mean
    density is given (rho_bar, Eq. gravitational_force). Returns (f, T) of the window
    itself, whose nodes are exact: each depends only on inputs within 3 * steps nodes.
    fields: (rho0, ux0, uy0, T0) of the whole domain."""
    ny, nx = np.asarray(fields[0]).shape
    pad = 3 * int(steps)
    xs = np.arange(x0 - pad, x1 + pad)
    ylo = 0 if (cfg["hydro_bc"][2] != 0 and y0 - pad <= 0) else y0 - pad
    yhi = ny if (cfg["hydro_bc"][3] != 0 and y1 + pad >= ny) else y1 + pad
    ys = np.arange(ylo, yhi)
    if cfg["hydro_bc"][0] != 0:
        raise ValueError("window_step expects a domain periodic in x")
    wcfg = dict(cfg)
    wcfg["nx"], wcfg["ny"] = len(xs), len(ys)
    wcfg["rho_bar_fixed"] = float(rho_bar)
    hb, tb = list(cfg["hydro_bc"]), list(cfg["thermal_bc"])
    wcfg["hydro_bc"] = [0, 0, hb[2] if ylo == 0 else 0, hb[3] if yhi == ny else 0]
    wcfg["thermal_bc"] = [0, 0, tb[2] if ylo == 0 else 0, tb[3] if yhi == ny else 0]
    for name in ("rho_w", "T_w", "T_dirichlet"):
        arrs = list(cfg.get(name) or [None] * 4)
        wcfg[name] = [None, None] + [None if a is None else np.asarray(a)[np.mod(xs, nx)] for a in arrs[2:]]
    sub = [np.asarray(a)[np.ix_(np.mod(ys, ny), np.mod(xs, nx))] for a in fields]
    o = Oracle(wcfg, *sub)
    o.step(steps)
    iy = slice(y0 - ylo, y1 - ylo)
    ix = slice(pad, pad + (x1 - x0))
    return o.f[:, iy, ix].copy(), o.T[iy, ix].copy()


def energy_rhs(cfg: dict, rho, ux, uy, T):
    """The FD operator L(T) of Eq. (energy-equation) at every node (for unit pins)."""
    P, keep = make_params(cfg)
    ny, nx = int(cfg["ny"]), int(cfg["nx"])
    arrs = [np.ascontiguousarray(v, dtype=np.float64).reshape(ny, nx) for v in (rho, ux, uy, T)]
    out = np.empty((ny, nx))
    lib().orc_energy_rhs(ctypes.byref(P), *[_p(a) for a in arrs], _p(out))
    return out


def matrices():
    m = np.empty(81); mi = np.empty(81)
    lib().orc_matrix(_p(m), _p(mi))
    return m.reshape(9, 9), mi.reshape(9, 9)


def tc(cfg: dict) -> float:
    P, _ = make_params(cfg)
    return lib().orc_tc(ctypes.byref(P))
