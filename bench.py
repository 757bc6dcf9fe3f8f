"""Benchmark of the fused coupled LBM + energy step on GB300.

Workload (synthetic, seeded): 2-D pool boiling on a 2048 x 4096 grid (x periodic, Zou-He
psi-based walls at y = 0 and y = ny-1, bottom heater strip of nx/5 at T_sat + 0.1 Tc,
adiabatic elsewhere, liquid pool below 2/3 of the height, +-1e-3 Tc temperature noise,
g = 3e-5, PR EOS a = 3/49, sigma = 0.103). One bench step = one time step of the whole
grid (one fused kernel launch). Metric: coupled LBM + energy MLUPS of the FP32 path
(populations stored as f_i - w_i rho_ref), with the FP64 path measured beside it.

Launch: python bench.py [--gpus N --steps K --warmup W]  (N > 1 under torch.distributed.run:
each rank advances its own replica; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 2048, 4096
SIGMA = 0.103  # Table 2, base mesh (a = 6.12e-2 = 3/49) at T_sat = 0.86 Tc
BYTES_PER_NODE = {"fp32": 80, "fp64": 160}  # read + write of 9 populations and T


def workload(precision: str, nx=NX, ny=NY, thermo="product"):
    import workloads as W
    a, b, R, omega = 3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344
    if thermo == "product":
        from paper_2201_04560_gb300 import ppl
        Tc = ppl.tc(a, b, R)
        rv, rl, _ = ppl.maxwell(a, b, R, omega, 0.86 * Tc)
    else:
        from oracle import thermo as th
        e = th.PR(a=a, b=b, R=R, omega=omega)
        Tc = e.Tc
        rv, rl, _ = th.maxwell(e, 0.86 * Tc)
    return W.pool_boiling(Tc, rv, rl, SIGMA, nx=nx, ny=ny, g=3e-5, precision=precision)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def snapshot(self):
        """One query, taken right before and right after the timed region, so that a timed
        region shorter than the sampling period still carries a clock record."""
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
            if r.returncode == 0 and r.stdout.strip():
                self.lines.append(r.stdout.strip().splitlines()[0])
        except (OSError, subprocess.TimeoutExpired):
            pass

    def start(self):
        self.snapshot()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.snapshot()
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "sampling": "nvidia-smi every 100 ms during the timed region, plus one query right before "
                            "and one right after it"}


def profile_record(name, key):
    """A figure from a committed ncu summary (profiles/<name>), if it was taken on the current
    kernel sources (their sha256 is recorded beside it), else None."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for f in rec["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        return rec[key] if h.hexdigest() == rec["sources_sha256"] else None
    except (OSError, KeyError, ValueError):
        return None


def kernel_traffic():
    """ncu DRAM bytes of one FP32 step launch at the bench size, if taken on the current kernel sources."""
    return profile_record("traffic.json", "traffic_bytes_per_launch")


# GB300's dense FP64 rate is 1.25 TFLOP/s nominal: 2 FP64 FMA thread-operations per SM per clock
# (152 SMs x 2.07 GHz x 2 x 2 flops); the FP64 step's roofline is its FP64-pipe instruction rate
FP64_OPS_PER_SM_CLOCK = 2.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def time_device(sim, steps, warmup, torch, min_warm_s=0.0):
    """Device time of `steps` fused steps (CUDA events on the launching stream), after `warmup`
    untimed steps, continued in chunks until min_warm_s seconds have passed (on a GPU that has been
    idle, the SM clock of a new context stayed ~4 % below its maximum for the first ~0.4 s of load)."""
    stream = torch.cuda.Stream()
    sim.set_stream(stream)
    t0 = time.perf_counter()
    sim.step_async(warmup)
    sim.sync()
    warm_steps = warmup
    while time.perf_counter() - t0 < min_warm_s:
        sim.step_async(64)
        sim.sync()
        warm_steps += 64
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sim.launch_count
    torch.cuda.synchronize()
    start.record(stream)
    sim.step_async(steps)
    end.record(stream)
    end.synchronize()
    sim.sync()
    return start.elapsed_time(end) / 1e3, sim.launch_count - l0, warm_steps


def host_cpu():
    """Model name and logical core count of the host that runs the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "arch": platform.machine()}


def cpu_oracle_sample(steps=3):
    """The FP64 C oracle, single-threaded, on the same workload for a few steps."""
    from oracle import oracle
    cfg, ic = workload("fp64", thermo="oracle")
    o = oracle.Oracle(cfg, *ic)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": NX * NY * steps / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "%dx%d pool boiling, %d FP64 steps, single-threaded C oracle" % (NX, NY, steps),
            **host_cpu()}


def fp64_roofline(mlups64, ach_gbs, hbm, peaks, torch):
    """FP64 step against GB300's FP64 pipe: FP64-pipe thread-instructions per node (ncu,
    profiles/fp64_pipe.json) x node updates per second, over the FP64 FMA rate measured on this
    device by a DFMA loop on every SM (ppl_fp64_rate); the nominal rate (2 per SM per clock at
    the maximum SM clock) is reported beside it."""
    from paper_2201_04560_gb300 import ppl
    per_node = profile_record("fp64_pipe.json", "fp64_pipe_thread_inst_per_node")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = FP64_OPS_PER_SM_CLOCK * sms * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = ppl.fp64_rate(4000)
    achieved = per_node * mlups64 * 1e6 if per_node else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FP64 thread-instr/s",
            "frac": achieved / peak if achieved else None,
            "peak_kind": "measured: DFMA loop on every SM (ppl_fp64_rate), FP64 FMA thread-operations per second",
            "nominal_peak": nominal, "nominal_frac": achieved / nominal if achieved else None,
            "achieved_gbs": ach_gbs, "hbm_frac": ach_gbs / hbm, "bytes_per_node": BYTES_PER_NODE["fp64"]}


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle
    # the crop shrinks with the step count so that the whole run stays near 80 s of CPU
    # (the oracle updates about 2.5 M nodes/s on one core)
    nodes = max(256 * 32, int(2.0e8 / (args.steps + args.warmup)))
    nx, ny = 256, max(32, min(NY, nodes // 256))
    cfg, ic = workload("fp64", nx=nx, ny=ny, thermo="oracle")
    o = oracle.Oracle(cfg, *ic)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = nx * ny * args.steps / dt / 1e6
    sample = "%dx%d crop of the pool-boiling workload, FP64 C oracle, single-threaded" % (nx, ny)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "pool boiling %dx%d, FP32 populations as f - w rho_ref" % (NX, NY), "grid": [NX, NY],
                   "sample": "%dx%d crop per step" % (nx, ny)},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample, **host_cpu()},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


METRIC = "coupled LBM+energy MLUPS (FP32 vs FP64, same GB300) and % of HBM roofline"


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over the ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, dt_max, world):
    """Replicas only: every rank advances its own copy of the workload, so the job's node
    updates are world x nodes x steps, over the slowest rank's time."""
    return world * nodes_per_rank * steps / dt_max / 1e6


def _json_ready(x):
    if isinstance(x, dict):
        return {str(k): _json_ready(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_json_ready(v) for v in x]
    if hasattr(x, "item"):
        return x.item()
    return x


# The paper's mesh-refinement studies (Secs. 4.1, 4.3): name -> (study, keyword arguments)
EXPERIMENTS = {
    # droplet vaporization, 128^2 / 256^2 / 512^2 with 1:4:16 steps, R = 40 on 256^2, 0.8 / 0.9 T_c,
    # kappa 0.3, lambda 0.25; D^2-law slope per mesh
    "droplet-refinement": ("droplet_vaporization_study", dict(meshes=(128, 256, 512), R0=20.0, coarse_steps=200000,
                                                               sample_every=500)),
    # Table 2: L = 128 ... 432 (ratio 1.5), T_sat 0.86 T_c, vapour at T_c, lambda 2/3, 0.4e6 steps
    "table2": ("droplet_vaporization_study", dict(meshes=(128, 192, 288, 432), R0=32.0, T_ratio=0.86,
                                                  Tv_ratio=1.0, lam=2.0 / 3.0, kappa=0.0, width=2.0 / 0.92,
                                                  coarse_steps=400000, sample_every=64)),
    # contact-angle table: psi-based model, rho_w = 4.0 / 2.3 / 1.7, meshes 160 ... 810
    "contact-psi": ("contact_angle_study", dict(meshes=(160, 240, 360, 540, 810))),
    # G_w table: modified psi-based model, G_w per mesh keeping the angle of G_w = -0.8 on 160^2
    "gw-search": ("G_w_search", dict()),
    # pool boiling, rho_wh = 3.44 and T_h = 1.2 T_c: d^N, D^N, Q(t), time shifts
    "pool-refinement": ("pool_boiling_study", dict()),
    # Table 3: the one-dimensional boiling-like problem, L = 160 ... 2560, both parameter sets
    "stefan-refinement": ("stefan_study", dict()),
    # the batched refinement sequence against stepping its handles one after another
    "batch-throughput": ("batch_throughput", dict()),
    # the FP32 path against the FP64 path, per field, on the four synthetic cases
    "fp32-error": ("fp32_error_study", dict()),
    # MLUPS and HBM fraction of the step on each synthetic case, FP32 and FP64
    "cases": ("bench.case_throughput", dict()),
    # sigma and kappa of the 192^2 mesh tuned on the lattice with sensitivity runs (Sec. 3.2)
    "calibration": ("calibration.calibrate_mesh", dict(n_base=128, n=192)),
}


def case_throughput():
    """Node updates per second of the fused step on the synthetic cases shaped like the paper's
    (the static droplet, the Stefan strip, the droplet in superheated vapour, pool boiling),
    FP32 and FP64, default launch shape and autotuned, with the fraction of the HBM roofline
    (80 / 160 algorithmic bytes per node over the measured copy bandwidth). The small cases fit
    in L2 and are launch- and latency-bound; only pool boiling is HBM-sized."""
    import torch
    import workloads as W
    from paper_2201_04560_gb300 import ppl
    a, b, R, om = 3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344
    Tc = ppl.tc(a, b, R)
    rv8, rl8, _ = ppl.maxwell(a, b, R, om, 0.8 * Tc)
    rv6, rl6, _ = ppl.maxwell(a, b, R, om, 0.86 * Tc)
    s86 = ppl.sigma_for(a, b, R, om, -1.0, 0.86 * Tc)
    cases = {
        "static droplet 64x64": lambda p: W.static_droplet(Tc, rv8, rl8, nx=64, ny=64, precision=p),
        "Stefan strip 1024x4": lambda p: W.stefan_strip(Tc, rv6, rl6, s86, nx=1024, ny=4, precision=p),
        "droplet vaporization 256x256": lambda p: W.droplet_vaporization(Tc, rv8, rl8, 0.1, nx=256, ny=256,
                                                                        R0=40.0, iso_steps=2000, precision=p),
        "pool boiling 1024x2048": lambda p: W.pool_boiling(Tc, rv6, rl6, SIGMA, nx=1024, ny=2048, g=3e-5,
                                                          precision=p),
    }
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    out = {}
    for name, make in cases.items():
        for prec in ("fp32", "fp64"):
            cfg, ic = make(prec)
            nodes = cfg["nx"] * cfg["ny"]
            steps = max(64, min(20000, int(2e10 / nodes / (1 if prec == "fp32" else 25))))
            with ppl.Simulation(cfg, *ic) as sim:
                if cfg["energy_on"]:
                    sim.step(cfg["iso_steps"])  # time the coupled step, past the isothermal start
                dt = time_device(sim, steps, 32, torch)[0]
                rec = {"kernel": sim.kernel, "rows": sim.launch()[0], "mlups": nodes * steps / dt / 1e6}
                rows, _ = sim.autotune(64)
                dt2 = time_device(sim, steps, 32, torch)[0]
                rec.update(autotuned_kernel=sim.kernel, autotuned_rows=rows, autotuned_mlups=nodes * steps / dt2 / 1e6)
            best = max(rec["mlups"], rec["autotuned_mlups"])
            rec["hbm_frac"] = best * 1e6 * BYTES_PER_NODE[prec] / 1e9 / hbm
            rec["steps"] = steps
            out["%s %s" % (name, prec)] = rec
    return out


def run_experiment(args):
    import importlib
    name = args.experiment
    fn, kw = EXPERIMENTS[name]
    mod, _, fname = fn.rpartition(".")
    if mod == "bench":
        study = globals()[fname]
    else:
        study = getattr(importlib.import_module("paper_2201_04560_gb300." + (mod or "refinement")), fname)
    kw = dict(kw)
    if args.coarse_steps and fname not in ("fp32_error_study", "batch_throughput", "case_throughput"):
        kw["coarse_steps"] = args.coarse_steps
    if args.precision in ("fp32", "fp64") and not mod and fname not in ("G_w_search", "fp32_error_study"):
        kw["precision"] = args.precision
    t0 = time.time()
    if name == "contact-psi":
        out = {"runs": [study(value=v, **kw) for v in (4.0, 2.3, 1.7)]}
    elif name == "stefan-refinement":
        out = {"runs": [study(param_set=k, **kw) for k in (1, 2)]}
    else:
        out = study(**kw)
    out = {"experiment": name, "wall_seconds": time.time() - t0, **out}
    print(json.dumps(_json_ready(out)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=32)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=0, help="FP64 timed steps (default steps/8, >= 8)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--precision", default="both", choices=["both", "fp32", "fp64"])
    ap.add_argument("--nx", type=int, default=NX, help="grid width (profiling runs; the bench workload is 2048)")
    ap.add_argument("--ny", type=int, default=NY, help="grid height (profiling runs; the bench workload is 4096)")
    ap.add_argument("--kernel", default="auto", choices=["auto", "column", "pair"],
                    help="FP32 step kernel (profiling runs; auto picks the two-column kernel where it applies)")
    ap.add_argument("--experiment", default=None, choices=sorted(EXPERIMENTS),
                    help="run one of the paper's mesh-refinement studies instead of the throughput step")
    ap.add_argument("--coarse-steps", type=int, default=0, help="experiment length in first-mesh steps")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.experiment:
        return run_experiment(args)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_2201_04560_gb300 import Simulation

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()


    nx, ny = args.nx, args.ny
    nodes = nx * ny
    peaks, peak_kind = measured_peaks()
    out = {}
    precs = ("fp32", "fp64") if args.precision == "both" else (args.precision,)
    for prec in precs:
        steps = args.steps if prec == "fp32" else (args.fp64_steps or max(8, args.steps // 8))
        cfg, ic = workload(prec, nx=nx, ny=ny)
        sim = Simulation(cfg, *ic)
        if prec == "fp32" and args.kernel != "auto":
            sim.select_kernel(args.kernel)
        sampler = ClockSampler(local) if prec == "fp32" else None
        barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        dt, launches, warm_steps = time_device(sim, steps, args.warmup, torch, min_warm_s=1.0 if prec == "fp32" else 0.0)
        clocks = sampler.stop() if sampler else None
        barrier()
        dt = max_over_ranks(dt, dist, "cuda")
        n = sim.norms()
        out[prec] = {"dt": dt, "steps": steps, "launches": launches, "clocks": clocks, "flags": n["flags"],
                     "mass": n["mass"], "kernel": sim.kernel, "rows_per_cta": sim.launch()[0],
                     "warm_steps": warm_steps,
                     "staging": "tma" if sim.tma_staging else "cp.async"}
        if prec == "fp32" and not args.no_e2e:
            # end to end through the C ABI: pinned host inputs -> device, K steps, fields -> host
            host_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory() for a in ic]
            host_out = [torch.empty((ny, nx), dtype=torch.float64).pin_memory() for _ in range(4)]
            import ctypes
            P = ctypes.POINTER(ctypes.c_double)
            sim.set_stream(None)
            barrier()
            t0 = time.perf_counter()
            rc = sim.lib.ppl_reset(sim.h, *[ctypes.cast(t.data_ptr(), P) for t in host_in])
            assert rc == 0, rc
            sim.step(steps)
            rc = sim.lib.ppl_fields(sim.h, *[ctypes.cast(t.data_ptr(), P) for t in host_out])
            assert rc == 0, rc
            e2e_dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
            out["e2e"] = {"value": whole_job_mlups(nodes, steps, e2e_dt, world), "unit": "MLUPS",
                          "h2d_bytes_per_step": int(4 * nodes * 8 / steps),
                          "d2h_bytes_per_step": int(4 * nodes * 8 / steps)}
        sim.close()
        del sim
        torch.cuda.empty_cache()

    if rank != 0:
        return
    if args.precision != "both" or args.no_e2e:
        # profiling / partial runs: timing summary only
        print(json.dumps({p: {"mlups": whole_job_mlups(nodes, v["steps"], v["dt"], world),
                              "ms_per_step": v["dt"] / v["steps"] * 1e3,
                              "kernel": v["kernel"], "rows_per_cta": v["rows_per_cta"]}
                          for p, v in out.items() if p in ("fp32", "fp64")}))
        return
    f32, f64 = out["fp32"], out["fp64"]
    mlups32 = whole_job_mlups(nodes, f32["steps"], f32["dt"], world)
    mlups64 = whole_job_mlups(nodes, f64["steps"], f64["dt"], world)
    per_launch32 = f32["dt"] / f32["steps"]
    per_launch64 = f64["dt"] / f64["steps"]
    ach32 = BYTES_PER_NODE["fp32"] * nodes / per_launch32 / 1e9
    ach64 = BYTES_PER_NODE["fp64"] * nodes / per_launch64 / 1e9
    hbm = float(peaks["hbm_gbs"])
    line = {
        "metric": METRIC,
        "value": mlups32, "unit": "MLUPS", "n_gpus": world, "steps": f32["steps"], "warmup": args.warmup,
        "ms_per_step": per_launch32 * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "pool boiling %dx%d, FP32 populations as f - w rho_ref" % (NX, NY),
                   "grid": [NX, NY], "l2": "state (335 MB FP32, 671 MB FP64 per buffer) larger than L2",
                   "parallelism": "replica per GPU" if world > 1 else "single GPU",
                   "kernel": {"fp32": f32["kernel"], "fp64": f64["kernel"]},
                   "rows_per_cta": {"fp32": f32["rows_per_cta"], "fp64": f64["rows_per_cta"]},
                   "fp32_row_staging": f32["staging"],
                   "warmup_rule": "at least --warmup untimed steps, continued until 1 s of untimed steps have run "
                                  "(a freshly started context runs its first ~0.4 s below the maximum SM clock); "
                                  "FP32 warm-up steps run: %d" % f32["warm_steps"]},
        "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s", "frac": ach32 / hbm,
                     "traffic": kernel_traffic(), "peak_kind": peak_kind, "bytes_per_node": BYTES_PER_NODE["fp32"]},
        "fp64": {"value": mlups64, "unit": "MLUPS", "steps": f64["steps"], "ms_per_step": per_launch64 * 1e3,
                 "roofline": fp64_roofline(mlups64, ach64, hbm, peaks, torch)},
        "e2e": out["e2e"],
        "gpu_launches": f32["launches"],
        "clocks": f32["clocks"],
        "status_flags": {"fp32": f32["flags"], "fp64": f64["flags"]},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
