"""ctypes binding of libppl (include/ppl.h): argument marshalling only.

Every step of the time integration runs in the sm_103a kernels of libppl.so. There is
no CPU fallback: if the library is missing or no CUDA device is present the calls
raise. PyTorch, when used, only supplies device buffers and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PPL_OK, PPL_E_INVAL, PPL_E_CUDA, PPL_E_NUMERIC, PPL_E_TIMEOUT, PPL_E_IO, PPL_E_NOMEM = 0, -1, -2, -3, -4, -5, -6
PPL_FP64, PPL_FP32DEV = 0, 1
PPL_FP64_DSIGMA, PPL_FP64_DKAPPA = 2, 3  # FP64 state + its derivative w.r.t. sigma / kappa
PPL_FP32_DSIGMA, PPL_FP32_DKAPPA = 4, 5  # the same in FP32 arithmetic and deviation storage
PRECISIONS = {"fp64": PPL_FP64, "fp32": PPL_FP32DEV, "fp64_dsigma": PPL_FP64_DSIGMA,
              "fp64_dkappa": PPL_FP64_DKAPPA, "fp32_dsigma": PPL_FP32_DSIGMA, "fp32_dkappa": PPL_FP32_DKAPPA}
FLAG_PSI_NEG, FLAG_NAN, FLAG_RHO_NONPOS, FLAG_STALL = 1, 2, 4, 8

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PU8 = ctypes.POINTER(ctypes.c_uint8)


class PplConfig(ctypes.Structure):
    """Mirror of ppl_config in include/ppl.h."""

    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("rho_ref", _D), ("T_ref", _D), ("a", _D), ("b", _D), ("R", _D), ("omega", _D), ("G", _D),
        ("s", _D * 9),
        ("eta_l", _D), ("eta_v", _D), ("rho_l", _D), ("rho_v", _D),
        ("sigma", _D), ("kappa", _D), ("gx", _D), ("gy", _D), ("cv", _D), ("lambda_l", _D), ("lambda_v", _D),
        ("energy_on", ctypes.c_int32), ("iso_steps", ctypes.c_int64),
        ("hydro_bc", ctypes.c_int32 * 4), ("thermal_bc", ctypes.c_int32 * 4),
        ("T_side", _D * 4), ("rho_w_side", _D * 4),
        ("rho_w", _PD * 4), ("T_w", _PD * 4), ("T_dirichlet", _PU8 * 4),
        ("contact_model", ctypes.c_int32), ("G_w", _D),
    ]


class PplNorms(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("mass", _D), ("rho_mean", _D), ("sum_abs_rho", _D),
                ("sum_abs_T", _D), ("rho_min", _D), ("rho_max", _D), ("T_min", _D), ("T_max", _D),
                ("flags", ctypes.c_uint32)]


class PplError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load_library().ppl_strerror(code).decode()
        super().__init__("%s: %s (code %d)" % (what, msg, code))


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libppl.so (building it in-tree with nvcc when it is missing or stale).

    The environment variable PPL_LIBRARY names another build of the library to load
    instead (no build step then)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("PPL_LIBRARY")
    if not path:
        if build_if_missing:
            _build.build_library()
        path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libppl.so is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    H = ctypes.c_void_p
    L.ppl_init.argtypes = [ctypes.POINTER(PplConfig), _PD, _PD, _PD, _PD, ctypes.POINTER(H)]
    L.ppl_reset.argtypes = [H, _PD, _PD, _PD, _PD]
    L.ppl_set_stream.argtypes = [H, ctypes.c_void_p]
    L.ppl_step.argtypes = [H, ctypes.c_int64]
    L.ppl_step_async.argtypes = [H, ctypes.c_int64]
    L.ppl_sync.argtypes = [H]
    L.ppl_fields.argtypes = [H, _PD, _PD, _PD, _PD]
    L.ppl_fields_device.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int]
    L.ppl_populations.argtypes = [H, _PD]
    L.ppl_state_device.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    L.ppl_state_device.restype = ctypes.c_int
    L.ppl_snapshot_bytes.argtypes = [H]
    L.ppl_snapshot_bytes.restype = ctypes.c_size_t
    L.ppl_snapshot.argtypes = [H, ctypes.c_void_p]
    L.ppl_snapshot.restype = ctypes.c_int
    L.ppl_restore.argtypes = [H, ctypes.c_void_p, ctypes.c_int64]
    L.ppl_restore.restype = ctypes.c_int
    L.ppl_adjoint_scratch_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    L.ppl_adjoint_scratch_bytes.restype = ctypes.c_size_t
    L.ppl_adjoint_step.argtypes = [ctypes.POINTER(PplConfig)] + [ctypes.c_void_p] * 7
    L.ppl_adjoint_step.restype = ctypes.c_int
    L.ppl_tangent_fields.argtypes = [H, _PD, _PD, _PD, _PD]
    L.ppl_tangent_fields.restype = ctypes.c_int
    L.ppl_norms.argtypes = [H, ctypes.POINTER(PplNorms)]
    L.ppl_save.argtypes = [H, ctypes.c_char_p]
    L.ppl_load.argtypes = [H, ctypes.c_char_p]
    L.ppl_launch_count.argtypes = [H]
    L.ppl_launch_count.restype = ctypes.c_int64
    L.ppl_destroy.argtypes = [H]
    L.ppl_destroy.restype = None
    L.ppl_strerror.argtypes = [ctypes.c_int]
    L.ppl_strerror.restype = ctypes.c_char_p
    L.ppl_tc.argtypes = [_D, _D, _D]
    L.ppl_tc.restype = _D
    L.ppl_maxwell.argtypes = [_D, _D, _D, _D, _D, _PD, _PD, _PD]
    L.ppl_step_noalloc.argtypes = [ctypes.POINTER(PplConfig)] + [ctypes.c_void_p] * 8
    L.ppl_step_noalloc.restype = ctypes.c_int
    L.ppl_sigma_for.argtypes = [_D] * 6 + [_PD]
    L.ppl_gamma_planar.argtypes = [_D] * 8 + [_PD]
    L.ppl_kappa_for.argtypes = [_D, ctypes.c_int32, ctypes.c_int32] + [_D] * 6 + [_PD]
    L.ppl_refine.argtypes = [ctypes.POINTER(PplConfig), ctypes.c_int32, ctypes.c_int32, _D, ctypes.POINTER(PplConfig)]
    for name in ("ppl_sigma_for", "ppl_gamma_planar", "ppl_kappa_for", "ppl_refine"):
        getattr(L, name).restype = ctypes.c_int
    L.ppl_pressure.argtypes = [_D] * 6 + [_PD, _PD]
    L.ppl_pressure.restype = ctypes.c_int
    L.ppl_refine_a.argtypes = [_D, ctypes.c_int32, ctypes.c_int32]
    L.ppl_refine_a.restype = _D
    L.ppl_cross_norm.argtypes = [H, H, ctypes.c_int, _PD, _PD]
    L.ppl_batch_create.argtypes = [ctypes.POINTER(H), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                   ctypes.POINTER(H)]
    L.ppl_batch_step.argtypes = [H, ctypes.c_int64]
    L.ppl_batch_destroy.argtypes = [H]
    L.ppl_batch_destroy.restype = None
    L.ppl_batch_set_mode.argtypes = [H, ctypes.c_int]
    L.ppl_batch_set_mode.restype = ctypes.c_int
    L.ppl_batch_get_mode.argtypes = [H]
    L.ppl_batch_get_mode.restype = ctypes.c_int
    L.ppl_batch_set_wait_limit.argtypes = [H, ctypes.c_int64]
    L.ppl_batch_set_wait_limit.restype = ctypes.c_int
    L.ppl_set_launch.argtypes = [H, ctypes.c_int32]
    L.ppl_get_launch.argtypes = [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.ppl_autotune.argtypes = [H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _PD]
    L.ppl_select_kernel.argtypes = [H, ctypes.c_int]
    L.ppl_select_kernel.restype = ctypes.c_int
    L.ppl_get_kernel.argtypes = [H]
    L.ppl_get_kernel.restype = ctypes.c_int
    L.ppl_tma_staging.argtypes = [H]
    L.ppl_tma_staging.restype = ctypes.c_int
    L.ppl_stall_probe.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)]
    L.ppl_stall_probe.restype = ctypes.c_int
    L.ppl_fp64_rate.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.ppl_fp64_rate.restype = ctypes.c_int
    L.ppl_phase_area.argtypes = [H, _D, _D, _PD]
    L.ppl_relative_change.argtypes = [_PD, _PD, ctypes.c_int64, _PD]
    L.ppl_wall_heat_flux.argtypes = [H, ctypes.c_int, _PD]
    L.ppl_contact_angle.argtypes = [_PD, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, _D, _PD]
    L.ppl_time_shift.argtypes = [H, H, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64), _PD]
    L.ppl_time_shift.restype = ctypes.c_int
    for name in ("ppl_phase_area", "ppl_relative_change", "ppl_wall_heat_flux", "ppl_contact_angle"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("ppl_init", "ppl_reset", "ppl_set_stream", "ppl_step", "ppl_step_async", "ppl_sync",
                 "ppl_fields", "ppl_fields_device", "ppl_populations", "ppl_norms", "ppl_save", "ppl_load",
                 "ppl_maxwell", "ppl_cross_norm", "ppl_batch_create", "ppl_batch_step", "ppl_set_launch",
                 "ppl_get_launch", "ppl_autotune"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != PPL_OK:
        raise PplError(rc, what)


def tc(a: float, b: float, R: float = 1.0) -> float:
    """Critical temperature of the PR EOS (ppl_tc)."""
    return load_library().ppl_tc(a, b, R)


def maxwell(a: float, b: float, R: float, omega: float, T: float):
    """Maxwell coexistence (rho_v, rho_l, p_sat) of the PR isotherm (ppl_maxwell)."""
    rv, rl, ps = _D(), _D(), _D()
    _check(load_library().ppl_maxwell(a, b, R, omega, T, ctypes.byref(rv), ctypes.byref(rl), ctypes.byref(ps)),
           "ppl_maxwell")
    return rv.value, rl.value, ps.value


def pressure(a, b, R, omega, T, rho):
    """(p, dp/drho) of the Peng-Robinson EOS (ppl_pressure)."""
    p, dp = _D(), _D()
    _check(load_library().ppl_pressure(a, b, R, omega, T, rho, ctypes.byref(p), ctypes.byref(dp)), "ppl_pressure")
    return p.value, dp.value


def stall_probe(limit_ns: int) -> int:
    """Status word left by one CTA waiting, with the step kernel's bounded mbarrier wait, on an
    mbarrier that nothing completes (ppl_stall_probe): FLAG_STALL after limit_ns."""
    flags = ctypes.c_uint32(0)
    _check(load_library().ppl_stall_probe(int(limit_ns), ctypes.byref(flags)), "ppl_stall_probe")
    return int(flags.value)


def fp64_rate(iters: int = 2000) -> float:
    """Measured FP64 FMA thread-operations per second of the current device (ppl_fp64_rate)."""
    r = ctypes.c_double(0.0)
    _check(load_library().ppl_fp64_rate(int(iters), ctypes.byref(r)), "ppl_fp64_rate")
    return float(r.value)


def refine_a(a_base: float, n_base: int, n: int) -> float:
    return load_library().ppl_refine_a(a_base, n_base, n)


def sigma_for(a, b, R, omega, G, T) -> float:
    """Sec. 3.2 sigma tuning (ppl_sigma_for)."""
    out = _D()
    _check(load_library().ppl_sigma_for(a, b, R, omega, G, T, ctypes.byref(out)), "ppl_sigma_for")
    return out.value


def gamma_planar(a, b, R, omega, G, T, sigma, kappa) -> float:
    """Planar surface tension (ppl_gamma_planar)."""
    out = _D()
    _check(load_library().ppl_gamma_planar(a, b, R, omega, G, T, sigma, kappa, ctypes.byref(out)),
           "ppl_gamma_planar")
    return out.value


def kappa_for(a_base, n_base, n, b, R, omega, G, T_ratio, kappa_base=0.0) -> float:
    """Kappa of a refined mesh (ppl_kappa_for)."""
    out = _D()
    _check(load_library().ppl_kappa_for(a_base, n_base, n, b, R, omega, G, T_ratio, kappa_base, ctypes.byref(out)),
           "ppl_kappa_for")
    return out.value


def refine(cfg: dict, n_base: int, n: int, T_ratio: float) -> dict:
    """The Sec. 3 refinement of a configuration dict (ppl_refine); per-node arrays must be absent."""
    C, keep = make_config(cfg)
    O = PplConfig()
    _check(load_library().ppl_refine(ctypes.byref(C), n_base, n, T_ratio, ctypes.byref(O)), "ppl_refine")
    out = dict(cfg)
    out.update(nx=O.nx, ny=O.ny, a=O.a, sigma=O.sigma, kappa=O.kappa, gx=O.gx, gy=O.gy, T_ref=O.T_ref,
               iso_steps=O.iso_steps,
               T_side=[O.T_side[i] for i in range(4)])
    return out


def _ptr(a):
    return a.ctypes.data_as(_PD)


def make_config(cfg: dict):
    """Marshal a config dict (schema of the workloads module) into ppl_config."""
    C = PplConfig()
    keep = []
    C.nx, C.ny = int(cfg["nx"]), int(cfg["ny"])
    prec = cfg.get("precision", "fp64")
    C.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    C.rho_ref = float(cfg.get("rho_ref", 1.0))
    C.T_ref = float(cfg.get("T_ref", 0.0))
    for k in ("a", "b", "R", "omega", "G", "eta_l", "eta_v", "rho_l", "rho_v", "sigma", "kappa", "gx", "gy",
              "cv", "lambda_l", "lambda_v"):
        setattr(C, k, float(cfg[k]))
    for i in range(9):
        C.s[i] = float(cfg["s"][i])
    C.energy_on = int(cfg["energy_on"])
    C.iso_steps = int(cfg["iso_steps"])
    for sd in range(4):
        C.hydro_bc[sd] = int(cfg["hydro_bc"][sd])
        C.thermal_bc[sd] = int(cfg["thermal_bc"][sd])
        C.T_side[sd] = float(cfg["T_side"][sd])
        C.rho_w_side[sd] = float(cfg["rho_w_side"][sd])
        for name, dt, ptr in (("rho_w", np.float64, _PD), ("T_w", np.float64, _PD), ("T_dirichlet", np.uint8, _PU8)):
            arr = (cfg.get(name) or [None] * 4)[sd]
            if arr is None:
                getattr(C, name)[sd] = ctypes.cast(None, ptr)
            else:
                a = np.ascontiguousarray(arr, dtype=dt)
                keep.append(a)
                getattr(C, name)[sd] = a.ctypes.data_as(ptr)
    C.contact_model = int(cfg.get("contact_model", 0))
    C.G_w = float(cfg.get("G_w", 0.0))
    return C, keep


def step_noalloc(cfg: dict, f_in, T_in, f_out, T_out, stats_in, stats_out, status, stream=None) -> int:
    """ppl_step_noalloc on caller-owned device buffers (integer device addresses, e.g.
    torch data_ptr()s): one step that allocates no device memory. Returns the ppl code."""
    C, keep = make_config(cfg)
    handle = getattr(stream, "cuda_stream", stream)
    ptrs = [ctypes.c_void_p(int(p)) for p in (f_in, T_in, f_out, T_out, stats_in, stats_out, status)]
    return load_library().ppl_step_noalloc(ctypes.byref(C), *ptrs, ctypes.c_void_p(handle or None))


def adjoint_scratch_bytes(nx: int, ny: int) -> int:
    return int(load_library().ppl_adjoint_scratch_bytes(int(nx), int(ny)))


def adjoint_step(cfg: dict, f, T, fbar_in, fbar_out, grad, scratch, stream=None):
    """ppl_adjoint_step on device buffers (integer device addresses, e.g. torch data_ptr()s):
    fbar_out = (d f^{n+1} / d f^n)^T fbar_in, grad[0:2] += d/d(sigma, kappa). Raises on error."""
    C, keep = make_config(cfg)
    handle = getattr(stream, "cuda_stream", stream)
    ptrs = [ctypes.c_void_p(int(p)) for p in (f, T, fbar_in, fbar_out, grad, scratch)]
    _check(load_library().ppl_adjoint_step(ctypes.byref(C), *ptrs, ctypes.c_void_p(handle or None)),
           "ppl_adjoint_step")


class Simulation:
    """One ppl handle: device-resident state advanced by the fused sm_103a step kernel."""

    def __init__(self, cfg: dict, rho0, ux0, uy0, T0, stream=None):
        self.lib = load_library()
        self.cfg = dict(cfg)
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self._c, self._keep = make_config(cfg)
        self.h = ctypes.c_void_p()
        arrs = self._host_fields(rho0, ux0, uy0, T0)
        _check(self.lib.ppl_init(ctypes.byref(self._c), *[_ptr(a) for a in arrs], ctypes.byref(self.h)), "ppl_init")
        if stream is not None:
            self.set_stream(stream)

    def _host_fields(self, *fields):
        return [np.ascontiguousarray(v, dtype=np.float64).reshape(self.ny, self.nx) for v in fields]

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (library stream)."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(self.lib.ppl_set_stream(self.h, ctypes.c_void_p(handle or None)), "ppl_set_stream")

    def reset(self, rho0, ux0, uy0, T0):
        arrs = self._host_fields(rho0, ux0, uy0, T0)
        _check(self.lib.ppl_reset(self.h, *[_ptr(a) for a in arrs]), "ppl_reset")

    def step(self, n: int = 1):
        _check(self.lib.ppl_step(self.h, int(n)), "ppl_step")

    def step_async(self, n: int = 1):
        _check(self.lib.ppl_step_async(self.h, int(n)), "ppl_step_async")

    def sync(self):
        _check(self.lib.ppl_sync(self.h), "ppl_sync")

    def fields(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        _check(self.lib.ppl_fields(self.h, *[_ptr(a) for a in out]), "ppl_fields")
        return dict(zip(("rho", "ux", "uy", "T"), out))

    def fields_device(self, torch_dtype=None):
        import torch
        dt = torch_dtype or torch.float64
        code = {torch.float64: 0, torch.float32: 1}[dt]
        out = [torch.empty((self.ny, self.nx), dtype=dt, device="cuda") for _ in range(4)]
        _check(self.lib.ppl_fields_device(self.h, *[ctypes.c_void_p(t.data_ptr()) for t in out], code),
               "ppl_fields_device")
        return dict(zip(("rho", "ux", "uy", "T"), out))

    def tangent_fields(self):
        """d(rho, u_x, u_y, T)/d(parameter) of a sensitivity simulation (fp64_d* / fp32_d*)."""
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        _check(self.lib.ppl_tangent_fields(self.h, *[_ptr(a) for a in out]), "ppl_tangent_fields")
        return dict(zip(("rho", "ux", "uy", "T"), out))

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        _check(self.lib.ppl_populations(self.h, _ptr(f)), "ppl_populations")
        return f

    def state_device(self, f, T):
        """FP64 absolute populations [9][ny][nx] and T [ny][nx] of the current state into two
        device buffers (integer addresses, e.g. torch data_ptr()s)."""
        _check(self.lib.ppl_state_device(self.h, ctypes.c_void_p(int(f)), ctypes.c_void_p(int(T))),
               "ppl_state_device")

    @property
    def snapshot_bytes(self) -> int:
        return int(self.lib.ppl_snapshot_bytes(self.h))

    def snapshot(self, dst):
        """Copy the stored state into a device buffer of snapshot_bytes (async on the stream)."""
        _check(self.lib.ppl_snapshot(self.h, ctypes.c_void_p(int(dst))), "ppl_snapshot")

    def restore(self, src, step: int):
        """Make a snapshot the current state, with the step counter set to `step`."""
        _check(self.lib.ppl_restore(self.h, ctypes.c_void_p(int(src)), int(step)), "ppl_restore")

    def norms(self):
        n = PplNorms()
        _check(self.lib.ppl_norms(self.h, ctypes.byref(n)), "ppl_norms")
        return {k: getattr(n, k) for k, _ in PplNorms._fields_}

    def save(self, path: str):
        _check(self.lib.ppl_save(self.h, os.fsencode(path)), "ppl_save")

    def load(self, path: str):
        _check(self.lib.ppl_load(self.h, os.fsencode(path)), "ppl_load")

    @property
    def launch_count(self) -> int:
        return int(self.lib.ppl_launch_count(self.h))

    def phase_area(self, rho_lo: float, rho_hi: float) -> float:
        """Liquid area in nodes: sum of clamp((rho - rho_lo) / (rho_hi - rho_lo), 0, 1)."""
        a = ctypes.c_double()
        _check(self.lib.ppl_phase_area(self.h, float(rho_lo), float(rho_hi), ctypes.byref(a)), "ppl_phase_area")
        return a.value

    def wall_heat_flux(self, side: int) -> float:
        """Mean heat flux entering through boundary line `side` (Eq. pool-heat-flux)."""
        q = ctypes.c_double()
        _check(self.lib.ppl_wall_heat_flux(self.h, int(side), ctypes.byref(q)), "ppl_wall_heat_flux")
        return q.value

    def set_launch(self, rows_per_cta: int = 0):
        """Rows per CTA of the step kernel (0 = default shape)."""
        _check(self.lib.ppl_set_launch(self.h, int(rows_per_cta)), "ppl_set_launch")

    KERNELS = {"auto": 0, "column": 1, "pair": 2}

    def select_kernel(self, kind: str = "auto"):
        """FP32 step kernel: "column" (one column per thread), "pair" (two columns per thread,
        packed f32x2; domains periodic in x for the flow, with even nx) or "auto"."""
        _check(self.lib.ppl_select_kernel(self.h, self.KERNELS[kind]), "ppl_select_kernel")

    @property
    def kernel(self) -> str:
        return {1: "column", 2: "pair"}[int(self.lib.ppl_get_kernel(self.h))]

    @property
    def tma_staging(self) -> bool:
        """The two-column FP32 step stages rows by TMA (strips off the periodic x seam)."""
        return bool(self.lib.ppl_tma_staging(self.h))

    def launch(self):
        """(rows per CTA, CTAs per step launch)."""
        r, c = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.ppl_get_launch(self.h, ctypes.byref(r), ctypes.byref(c)), "ppl_get_launch")
        return r.value, c.value

    def autotune(self, steps: int = 64):
        """Time the candidate launch shapes, keep the fastest; returns (rows, ms per step)."""
        r, ms = ctypes.c_int32(), ctypes.c_double()
        _check(self.lib.ppl_autotune(self.h, int(steps), ctypes.byref(r), ctypes.byref(ms)), "ppl_autotune")
        return r.value, ms.value

    def close(self):
        if self.h:
            self.lib.ppl_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def cross_norm(coarse: Simulation, fine: Simulation, field: str = "rho"):
    """(num, den) of the cross-grid L1 difference, Eqs. (rel-diff-timestep), (global-rel-diff):
    the coarse field interpolated bilinearly onto the fine nodes; num/den is the relative one."""
    code = {"rho": 0, "T": 1}[field]
    num, den = ctypes.c_double(), ctypes.c_double()
    _check(coarse.lib.ppl_cross_norm(coarse.h, fine.h, code, ctypes.byref(num), ctypes.byref(den)),
           "ppl_cross_norm")
    return num.value, den.value


BATCH_MODES = {"graph": 0, "persistent": 1, "auto": 2}


class Batch:
    """Handles advanced together, handle k by substeps[k] steps per outer step (Sec. 3:
    dt ~ dx^2). mode "graph": the grids run concurrently as the branches of one CUDA graph;
    "persistent": one persistent launch (captured in a CUDA graph) takes the tiles of every
    mesh's steps from a ticket counter (FP32 two-column handles only); "auto" (default): the
    persistent launch where it applies and no handle has gravity, else the graph."""

    def __init__(self, sims, substeps, mode: str = "auto"):
        if len(sims) != len(substeps):
            raise ValueError("one substep count per simulation")
        self.lib = load_library()
        self.sims = list(sims)  # keeps the handles alive while the batch exists
        hs = (ctypes.c_void_p * len(sims))(*[s.h.value for s in sims])
        subs = (ctypes.c_int32 * len(sims))(*[int(k) for k in substeps])
        self.b = ctypes.c_void_p()
        _check(self.lib.ppl_batch_create(hs, subs, len(sims), ctypes.byref(self.b)), "ppl_batch_create")
        if mode != "auto":
            self.set_mode(mode)

    def set_mode(self, mode: str):
        _check(self.lib.ppl_batch_set_mode(self.b, BATCH_MODES[mode]), "ppl_batch_set_mode")

    @property
    def mode(self) -> str:
        return {v: k for k, v in BATCH_MODES.items()}[int(self.lib.ppl_batch_get_mode(self.b))]

    def set_wait_limit(self, ns: int):
        """Bound of every dependency wait of the persistent launch, in nanoseconds."""
        _check(self.lib.ppl_batch_set_wait_limit(self.b, int(ns)), "ppl_batch_set_wait_limit")

    def step(self, outer: int = 1):
        _check(self.lib.ppl_batch_step(self.b, int(outer)), "ppl_batch_step")

    def close(self):
        if self.b:
            self.lib.ppl_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def relative_change(R, R_star) -> float:
    """Eq. (relative-change-R) of two equally sampled series (the library's host routine)."""
    a = np.ascontiguousarray(R, dtype=np.float64)
    b = np.ascontiguousarray(R_star, dtype=np.float64)
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("two 1-D series of one length")
    out = ctypes.c_double()
    _check(load_library().ppl_relative_change(_ptr(a), _ptr(b), len(a), ctypes.byref(out)), "ppl_relative_change")
    return out.value


def contact_angle(rho, side: int, rho_mid: float) -> float:
    """Contact angle in degrees of a droplet on boundary line `side` of a host density field
    (the library's host routine, ppl_contact_angle)."""
    a = np.ascontiguousarray(rho, dtype=np.float64)
    out = ctypes.c_double()
    _check(load_library().ppl_contact_angle(_ptr(a), a.shape[1], a.shape[0], int(side), float(rho_mid),
                                            ctypes.byref(out)), "ppl_contact_angle")
    return out.value


def time_shift(coarse: Simulation, finest: Simulation, m: int, stride: int, field: str = "rho"):
    """Eq. (rel-diff-minimize): (delta, minimum numerator) with `coarse` at tau - m and
    `finest` at tau; advances `coarse` through the search window (ppl_time_shift)."""
    d, num = ctypes.c_int64(), ctypes.c_double()
    _check(coarse.lib.ppl_time_shift(coarse.h, finest.h, {"rho": 0, "T": 1}[field], int(m), int(stride),
                                     ctypes.byref(d), ctypes.byref(num)), "ppl_time_shift")
    return d.value, num.value
