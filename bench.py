"""Benchmark of the coupled phase-field / surfactant / flow LBM step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]
                    [--workload shear|batch|warmstart|shear-track|conv] [--precision fp32|fp16|bf16]

Workload (default): the sheared sessile drop (top wall at u_w = 0.01, 90 deg contact
angle, psi0 = 0.02, solid-gas adsorption 0.5, tau = 0.8, eps = 4, FP32) on a
4096 x 2048 grid with R = 480, i.e. the 512 x 256 shear configuration scaled to the
domain size the throughput target is quoted on.  One step = one time step of the whole
coupled update over the whole grid (one kernel launch).  The 4096 x 2048 state
(2.2 GB) is far larger than the 126 MB L2, so no flush is needed between steps.

Workload 'batch': 512 sessile-drop instances of uneven seeded grids (64 x 32 to
512 x 256, contact angle, surfactant load and adsorption strengths drawn per
instance), all stepped by one persistent tile-queue launch per step replayed from a
CUDA graph, tiling chosen by the autotuner; the same instances stepped one launch
per instance per step are timed beside it.

Workload 'warmstart': the learned warm start on 256 x 128 sessile drops.  Training
drops (seeded parameters: contact angle U[30,150] deg, psi0 U[0.005,0.05], adsorption
strengths U[0,1], radius U[0.25,0.35] ny) are relaxed from cold starts by the batch
solver, the encoder-decoder is trained on the relaxed fields with the tensor-core
kernels, and held-out drops are relaxed from cold and from warm starts; the value is
the median ratio of cold to warm steps to equilibrium.

Workload 'shear-track': the 512 x 256 shear configuration run to 50,000 steps for three
solid-gas adsorption strengths (one batch), tracking the wetted segment on the wall.

Workload 'drop1000': a surfactant-laden drop at rest at the paper's density and viscosity
ratios (1000 and 100) on the same grid: the variable-property specialisation of the
step.  Option --multiplier exact adds the exact discrete multiplier's reduction pass
to every step of the shear or drop workload.

Workload 'conv': throughput of the warm-start network's tensor-core convolutions
(forward, input gradient, weight gradient) on its heaviest layers, against the BF16
tensor peak.

Prints one JSON line (rank 0).  Metric: MLUPS (million lattice-node updates per
second, whole job).  Under torchrun with N > 1 every rank steps its own replica of the
workload ('replicas only': the single-domain path has no multi-GPU exchange here).
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2609_26332_b300 import ranks  # noqa: E402

BYTES_PER_CELL = {"fp32": 264, "fp16": 132, "bf16": 132}   # algorithmic bytes per cell update
# the exact multiplier's reduction pass reads the phi set's 8 deviation planes, its
# float-float zeroth moment and phi^n once per cell
EXACT_BYTES_PER_CELL = {"fp32": 44, "fp16": 28, "bf16": 28}

# DRAM bytes (read + write) per step_kernel launch on the 4096 x 2048 shear workload from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), keyed by a hash of the
# step kernel's code and of the host code that splits the grid among the CTAs (comments
# stripped) and the float flags: a changed kernel or split reports null until re-measured.
TRAFFIC = {"ce6eb7d023f6123a": {"fp32": 2.398e9, "fp16": 1.346e9, "bf16": 1.348e9}}


def code_only(src):
    """CUDA source without comments and with whitespace collapsed: comments and layout do
    not change the kernel the counters were taken on."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_hash():
    import hashlib
    from paper_2609_26332_b300 import build as _b
    h = hashlib.sha256()
    for f in ("surflbm_step.cuh", "surflbm_step_tile.inc", "surflbm_device.cuh", "surflbm_api.cu"):
        h.update(code_only(open(os.path.join(_b.CSRC, f)).read()).encode())
    h.update(" ".join(_b.FLOAT_FLAGS).encode())
    return h.hexdigest()[:16]


def state_bytes_per_cell(precision):
    """Resident state: two buffers of 25 population planes, two float-float zeroth moments
    and phi of the previous step, plus six history planes in place."""
    es = 4 if precision == "fp32" else 2
    return 2 * (25 * es + 16 + 4) + 6 * es


DTYPE = {"fp32": "f32", "fp16": "f16-storage/f32-compute", "bf16": "bf16-storage/f32-compute"}


# the shear configuration's physics: Ca = mu u_w / sigma = 0.5 with tau = 0.8, u_w = 0.01
# (sigma = 0.002), Pi = 1.35, Ex = 0.5 as in the paper's Couette case (Sec. 4.5)
SHEAR_SIGMA, SHEAR_EX, SHEAR_PI = 0.002, 0.5, 1.35


def shear_case(nx, ny, precision="fp32"):
    R = 480.0 * ny / 2048.0
    return dict(nx=nx, ny=ny, R=R, xc=nx / 4.0, theta=90.0, psi0=0.02, beta_sg=0.5, beta_sl=0.0, u_w=0.01,
                precision=precision)


def drop1000_case(nx, ny, precision="fp32"):
    """A surfactant-laden drop at rest at the paper's density and viscosity ratios (Sec. 4.2:
    rho_l / rho_g = 1000, mu_l / mu_g = 100, sigma_gl,0 = 0.001, W = 0.24 and k_B T = 0.162
    relative to beta, i.e. Ex = 0.5, Pi = 1.35): the variable-property specialisation of the
    step on the benchmark grid, neutral no-slip walls."""
    return dict(nx=nx, ny=ny, R=0.25 * ny, xc=nx / 2.0, theta=90.0, psi0=0.01, beta_sg=0.0, beta_sl=0.0, u_w=0.0,
                precision=precision, init="free", sigma=0.001, rho_l=1000.0, rho_g=1.0, tau_f=0.53, tau_f_gas=0.8)


def init_fields(case):
    from paper_2609_26332_b300 import inputs
    pb = inputs.bulk_phi(case["psi0"], SHEAR_EX)
    if case.get("init") == "free":
        return inputs.free_drop(case["nx"], case["ny"], case["R"], 4.0, phi_b=pb, psi0=case["psi0"])
    return inputs.sessile_drop(case["nx"], case["ny"], case["R"], 4.0, xc=case["xc"], phi_b=pb, psi0=case["psi0"])


def step_config(args, case, world):
    """The `config` object of the single-domain workloads (both arms report the same)."""
    cells = args.nx * args.ny
    workload = ((f"shear-drop {args.nx}x{args.ny} R={case['R']:.0f} {args.precision} "
                 "(512x256 shear configuration scaled to the 4096x2048 target size)")
                if args.workload == "shear" else
                (f"surfactant drop at rest {args.nx}x{args.ny} R={case['R']:.0f} {args.precision}, "
                 "rho_l/rho_g = 1000, mu_l/mu_g = 100 (variable-property step)"))
    if args.multiplier != "paper":
        workload += f", {args.multiplier} multiplier"
    return {"workload": workload, "nx": args.nx, "ny": args.ny, "cells": cells, "parallelism": f"replicas{world}",
            "multiplier": args.multiplier,
            "l2": f"state {cells * state_bytes_per_cell(args.precision) / 1e9:.2f} GB >> 126 MB L2, no flush"}


def make_domain(case, stream):
    from paper_2609_26332_b300 import binding as B
    mult = {"paper": B.PAPER, "target": B.TARGET, "exact": B.EXACT}[case.get("multiplier", "paper")]
    extra = {k: case[k] for k in ("rho_l", "rho_g", "tau_f", "tau_f_gas") if k in case}
    p = B.default_params(case["nx"], case["ny"], precision=case["precision"], psi_b=case["psi0"],
                         sigma=case.get("sigma", SHEAR_SIGMA), Ex=SHEAR_EX, Pi=SHEAR_PI, multiplier=mult, **extra)
    d = B.Domain(p, stream=stream)
    d.set_wall(0, case["theta"], case["beta_sg"], case["beta_sl"], 0.0)
    d.set_wall(1, 90.0, 0.0, 0.0, case["u_w"])
    return d


class _NvmlLib:
    """The few read-only NVML queries the clock sampler needs, through the driver's
    libnvidia-ml directly (ctypes), for hosts without the Python NVML package."""

    NVML_CLOCK_SM = 1

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.L = ctypes.CDLL("libnvidia-ml.so.1")
        if self.L.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")

    def _handle(self, fn, arg):
        h = self.ct.c_void_p()
        if fn(arg, self.ct.byref(h)) != 0:
            raise RuntimeError("no NVML handle")
        return h

    def nvmlDeviceGetHandleByPciBusId(self, bus):
        return self._handle(self.L.nvmlDeviceGetHandleByPciBusId_v2, self.ct.c_char_p(bus))

    def nvmlDeviceGetHandleByIndex(self, i):
        return self._handle(self.L.nvmlDeviceGetHandleByIndex_v2, self.ct.c_uint(i))

    def _uint(self, fn, h, kind):
        v = self.ct.c_uint()
        if fn(h, self.ct.c_int(kind), self.ct.byref(v)) != 0:
            raise RuntimeError("NVML clock query failed")
        return v.value

    def nvmlDeviceGetClockInfo(self, h, kind):
        return self._uint(self.L.nvmlDeviceGetClockInfo, h, kind)

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        return self._uint(self.L.nvmlDeviceGetMaxClockInfo, h, kind)

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.ct.c_ulonglong()
        fn = getattr(self.L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.L.nvmlDeviceGetCurrentClocksThrottleReasons
        if fn(h, self.ct.byref(v)) != 0:
            raise RuntimeError("NVML reasons query failed")
        return v.value


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled DURING the timed region: an NVML
    polling thread every 5 ms (the Python NVML package, else the driver's libnvidia-ml
    through ctypes; one sample is also taken at start and at stop, so a region of a few
    milliseconds still has a record), else nvidia-smi at its 50 ms floor."""

    REASONS = (("hw_slowdown", "nvmlClocksEventReasonHwSlowdown", 0x8),
               ("hw_thermal_slowdown", "nvmlClocksEventReasonHwThermalSlowdown", 0x40),
               ("sw_thermal_slowdown", "nvmlClocksEventReasonSwThermalSlowdown", 0x20),
               ("sw_power_cap", "nvmlClocksEventReasonSwPowerCap", 0x4))
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_s=0.005):
        self.rows, self.proc, self.nvml, self.thread = [], None, None, None
        self.period = period_s
        try:
            import threading
            try:
                import pynvml
                pynvml.nvmlInit()
            except ImportError:
                pynvml = _NvmlLib()
            self.nvml = pynvml
            self.h = self._handle(pynvml, index)
            self.max_mhz = float(pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM))
            self.bits = [(name, getattr(pynvml, attr, bit)) for name, attr, bit in self.REASONS]
            self._sample()
            self.halt = threading.Event()
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            return
        except Exception:
            self.nvml = None
        try:
            self.path = tempfile.mktemp(suffix=".csv")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    @staticmethod
    def _handle(pynvml, index):
        """The NVML handle of torch's device `index` (matched by PCI bus id: NVML counts every
        GPU of the machine, CUDA only the visible ones)."""
        try:
            import torch
            pr = torch.cuda.get_device_properties(index)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
            return pynvml.nvmlDeviceGetHandleByPciBusId(bus.encode())
        except Exception:
            return pynvml.nvmlDeviceGetHandleByIndex(index)

    def _sample(self):
        n = self.nvml
        sm = float(n.nvmlDeviceGetClockInfo(self.h, n.NVML_CLOCK_SM))
        try:
            mask = n.nvmlDeviceGetCurrentClocksEventReasons(self.h)
        except Exception:
            mask = n.nvmlDeviceGetCurrentClocksThrottleReasons(self.h)
        self.rows.append((sm, [name for name, bit in self.bits if mask & bit]))

    def _loop(self):
        while not self.halt.wait(self.period):
            try:
                self._sample()
            except Exception:
                return

    def stop(self):
        if self.nvml is not None:
            self.halt.set()
            self.thread.join(timeout=2)
            try:
                self._sample()
            except Exception:
                pass
            sm = [r[0] for r in self.rows]
            reasons = sorted({x for r in self.rows for x in r[1]})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.rows), "source": "nvml, 5 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi, 50 ms"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        j = json.load(open(path))
        return float(j["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def measured_bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s): the burst figure (kernels timed alone)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        j = json.load(open(path))
        if "bf16_tflops" in j:
            return float(j["bf16_tflops"]), "measured"
    return 1800.0, "fallback"


def cpu_baseline(seconds=12.0):
    """The FP64 oracle, as it stands, on a bounded sample: the 512 x 256 shear configuration."""
    from oracle import Oracle, OracleParams, Wall
    case = shear_case(512, 256)
    phi0, psi0 = init_fields(case)
    p = OracleParams(nx=512, ny=256, psi_b=case["psi0"], sigma=SHEAR_SIGMA, Ex=SHEAR_EX, Pi=SHEAR_PI,
                     walls=[Wall(case["theta"], case["beta_sg"], case["beta_sl"], 0.0), Wall(90.0, 0, 0, case["u_w"])])
    o = Oracle(p, phi0, psi0)
    o.step(1)
    t = time.perf_counter()
    n = 0
    while time.perf_counter() - t < seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t
    return {"value": 512 * 256 * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"numpy FP64 oracle, 512x256 shear configuration, {n} steps, 1 thread"}


def run_reference(args, rank, world):
    """The oracle, as it stands, on the arm's own workload (the full nx x ny grid of the
    shear configuration).  numpy has nothing to warm up, so one untimed step stands for the
    warm-up; the timed steps stop early once 150 s have passed (a bounded sample of the K
    steps: the per-step time is what the value is made of)."""
    if rank != 0:
        return
    from oracle import Oracle, OracleParams, Wall
    case = shear_case(args.nx, args.ny, args.precision)
    phi0, psi0 = init_fields(case)
    p = OracleParams(nx=args.nx, ny=args.ny, psi_b=case["psi0"], sigma=SHEAR_SIGMA, Ex=SHEAR_EX, Pi=SHEAR_PI,
                     walls=[Wall(case["theta"], case["beta_sg"], case["beta_sl"], 0.0), Wall(90.0, 0, 0, case["u_w"])])
    o = Oracle(p, phi0, psi0)
    o.step(1)
    t = time.perf_counter()
    n = 0
    while n < args.steps and (n == 0 or time.perf_counter() - t < 150.0):
        o.step(1)
        n += 1
    dt = time.perf_counter() - t
    v = args.nx * args.ny * n / dt / 1e6
    sample = (f"numpy FP64 oracle, {n} of the {args.steps} timed steps of the {args.nx}x{args.ny} shear workload "
              f"itself (capped at 150 s), 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": "coupled-step MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / n * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(args, case, world),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args, rank, world, dist):
    """Aggregate MLUPS of the 512-instance batch: one graph-replayed tile-queue launch per
    step against per-instance launches of the same instances."""
    import ctypes
    import torch
    from paper_2609_26332_b300 import binding as B, inputs
    # weak scaling over one global list: `instances` drops per rank, drawn as one seeded list
    # of instances x world, each rank stepping its contiguous share (balanced by cells)
    specs_all = inputs.batch_instances(args.instances * world, seed=inputs.DEFAULT_SEED)
    lo, hi = ranks.instance_share([sp["nx"] * sp["ny"] for sp in specs_all], rank, world)
    specs = specs_all[lo:hi]
    cells_all = sum(sp["nx"] * sp["ny"] for sp in specs_all)
    params, walls, fields = [], [], []
    for sp in specs:
        pb = inputs.bulk_phi(sp["psi0"], 1.0)
        params.append(B.default_params(sp["nx"], sp["ny"], precision=args.precision, psi_b=sp["psi0"]))
        walls.append(((sp["theta0"], sp["beta_sg"], sp["beta_sl"], 0.0), (90.0, 0.0, 0.0, 0.0)))
        fields.append(inputs.sessile_drop(sp["nx"], sp["ny"], sp["R"], 4.0, phi_b=pb, psi0=sp["psi0"]))
    cells = sum(sp["nx"] * sp["ny"] for sp in specs)
    stream = torch.cuda.Stream()        # a capturable (non-default) stream for the graph
    b = B.Batch(params, walls, stream=stream)
    for i, (phi, psi) in enumerate(fields):
        b.init_fields(i, phi, psi)
    cache = args.tiling_cache or os.path.join(tempfile.gettempdir(), "surflbm_tiling.json")
    band_rows, ctas = b.autotune(cache)
    b.set_tiling(band_rows, ctas, args.graph_steps)
    strip_width = b.tiling()[0]
    b.step(args.warmup)
    torch.cuda.synchronize()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = timed(lambda: b.step(args.steps))
    clocks = sampler.stop() if sampler else None
    ms_batch = ranks.max_over_ranks(ms, dist, "cuda")

    # the same instances, one launch per instance per step
    k_inst = max(1, args.steps // 4)
    torch.cuda.synchronize()
    ms_inst = timed(lambda: [b.step_instance(i, k_inst) for i in range(len(specs))])
    ms_inst = ranks.max_over_ranks(ms_inst, dist, "cuda")

    # end to end: upload every instance from pinned host memory, step, read every field back
    pinned = [(torch.from_numpy(p).pin_memory().numpy(), torch.from_numpy(q).pin_memory().numpy())
              for p, q in fields]
    outs = [{k: torch.empty((sp["ny"], sp["nx"]), dtype=torch.float64).pin_memory().numpy()
             for k in ("phi", "psi", "ux", "uy", "p")} for sp in specs]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i, (p, q) in enumerate(pinned):
        b.init_fields(i, p, q)
    b.step(args.steps)
    for i in range(len(specs)):
        B.lib.slbm_batch_read_fields(b._h, i, *[outs[i][k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                                 for k in ("phi", "psi", "ux", "uy", "p")])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = ranks.max_over_ranks(e2e_s, dist, "cuda")
    tot_bad = sum(int(b.read_totals(i, check=False)["range_count"]) for i in range(len(specs)))

    if rank == 0:
        peak, peak_kind = measured_peaks()
        per_step_s = ms_batch / 1e3 / args.steps
        achieved = BYTES_PER_CELL[args.precision] * cells / per_step_s / 1e9
        value = cells_all * args.steps / (ms_batch / 1e3) / 1e6
        per_inst = cells_all * k_inst / (ms_inst / 1e3) / 1e6
        sizes = sorted({(sp["nx"], sp["ny"]) for sp in specs})
        line = {
            "metric": "batched coupled-step aggregate MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": {"workload": f"batch of {len(specs)} sessile drops, grids {sizes[0][0]}x{sizes[0][1]} to "
                                   f"{sizes[-1][0]}x{sizes[-1][1]}, theta0 U[30,150], psi0 U[0.005,0.05], "
                                   f"adsorption U[0,1], {args.precision}",
                       "instances": len(specs_all), "cells": cells_all, "rank0_share": [lo, hi],
                       "strip_width": strip_width, "band_rows": band_rows, "ctas_per_sm": ctas,
                       "cells_per_thread_per_piece": band_rows // 4,
                       "graph_steps": args.graph_steps, "parallelism": f"instance shares x{world}",
                       "l2": f"state {cells * 2 * BYTES_PER_CELL[args.precision] / 2 / 1e9:.1f} GB >> 126 MB L2, no flush"},
            "per_instance_launches": {"value": per_inst, "unit": "MLUPS", "steps": k_inst,
                                      "launches": k_inst * len(specs), "speedup_batched": value / per_inst},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         # the batch kernel's DRAM counters were taken on an earlier build
                         "traffic": None,
                         "peak_kind": peak_kind, "bytes_per_cell": BYTES_PER_CELL[args.precision],
                         "kernel_hash": kernel_hash()},
            "e2e": {"value": cells_all * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": 16 * cells_all / args.steps, "d2h_bytes_per_step": 40 * cells_all / args.steps},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "range_count": tot_bad,
        }
        print(json.dumps(line))
    b.close()


def run_warmstart(args, rank, world, dist):
    """Steps to equilibrium, cold vs learned warm start, on held-out drops."""
    import torch
    from paper_2609_26332_b300 import binding as B, warmstart as WS
    ny, nx = 128, 256
    t0 = time.perf_counter()
    logs = []
    log = lambda m: (logs.append(m), print(m, file=sys.stderr, flush=True))
    net = B.WarmStartNet(ny, nx, max_batch=args.ws_batch, seed=7 + rank)
    train_specs = WS.drop_specs(args.ws_train, seed=1000 + rank, ny=ny, nx=nx)
    test_specs = WS.drop_specs(args.ws_eval, seed=9000 + rank, ny=ny, nx=nx)
    cond, targets, steps, lbm_launches = WS.build_dataset(net, train_specs, args.ws_tol, args.ws_max_steps, log=log)
    t_data = time.perf_counter() - t0
    ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev[0].record()
    hist = WS.train(net, cond, targets, args.ws_epochs, args.ws_batch, args.ws_lr, log=log)
    ev[1].record()
    torch.cuda.synchronize()
    t_train = ev[0].elapsed_time(ev[1]) / 1e3
    t1 = time.perf_counter()
    res = WS.evaluate(net, test_specs, args.ws_eval_tol, args.ws_max_steps)
    t_eval = time.perf_counter() - t1
    both = (res["steps_cold"] > 0) & (res["steps_warm"] > 0)
    ratio = res["steps_cold"][both] / np.maximum(res["steps_warm"][both], 1)
    dang = np.abs(res["angle_cold"] - res["angle_warm"])[both]
    # training throughput of the conv kernels: 3 x forward FLOPs per sample (fwd, dgrad, wgrad)
    fwd_flops = sum(2 * 9 * ci * co * (ny >> lv) * (nx >> lv)
                    for lv, ci, co in [(0, 16, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 128),
                                       (2, 128, 128), (3, 128, 128), (3, 128, 128), (2, 256, 128), (2, 128, 128),
                                       (1, 192, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32)])
    train_tflops = 3 * fwd_flops * len(cond) * args.ws_epochs / t_train / 1e12
    if rank == 0:
        line = {
            "metric": "steps-to-equilibrium ratio, cold / learned warm start", "value": float(np.median(ratio))
            if len(ratio) else None, "unit": "x", "n_gpus": world, "steps": args.ws_epochs, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-conv/f32-lbm",
            "data": "synthetic: LBM-relaxed seeded sessile drops",
            "config": {"workload": f"warm start, {ny}x{nx} drops, {args.ws_train} training drops relaxed to "
                                   f"residual {args.ws_tol:g}, {args.ws_eval} held-out drops relaxed to "
                                   f"residual {args.ws_eval_tol:g} from cold and warm starts",
                       "train_converged": int(len(cond)), "train_diverged": int((steps == -2).sum()),
                       "train_unconverged": int((steps == -1).sum()), "epochs": args.ws_epochs,
                       "batch": args.ws_batch},
            "eval": {"pairs": int(both.sum()), "cold_converged": int((res["steps_cold"] > 0).sum()),
                     "warm_converged": int((res["steps_warm"] > 0).sum()),
                     "median_steps_cold": float(np.median(res["steps_cold"][both])) if both.any() else None,
                     "median_steps_warm": float(np.median(res["steps_warm"][both])) if both.any() else None,
                     "ratio_p25": float(np.quantile(ratio, 0.25)) if len(ratio) else None,
                     "angle_diff_median_deg": float(np.median(dang)) if len(dang) else None,
                     "angle_diff_max_deg": float(np.max(dang)) if len(dang) else None,
                     "frac_within_0p5deg": float(np.mean(dang < 0.5)) if len(dang) else None,
                     "accepted": int(res["accepted"].sum()),
                     "cold_steps": res["steps_cold"].tolist(), "warm_steps": res["steps_warm"].tolist(),
                     "cold_angles": [None if not np.isfinite(a) else round(float(a), 3) for a in res["angle_cold"]],
                     "warm_angles": [None if not np.isfinite(a) else round(float(a), 3) for a in res["angle_warm"]],
                     "theta0": [round(s["theta0"], 2) for s in test_specs]},
            "train": {"final_loss": hist[-1], "first_loss": hist[0], "seconds": t_train,
                      "conv_tflops": train_tflops},
            "seconds": {"dataset": t_data, "train": t_train, "eval": t_eval},
            # kernels per training step: input 1, convs 14, pools 3, upsample-concats 3, head 1,
            # input gradients 13, upsample / pool adjoints 6, weight and bias gradients 28,
            # Adam 1, weight refresh 14; per LBM step one batch launch
            "gpu_launches": int(84 * args.ws_epochs * max(1, len(cond) // args.ws_batch)
                                + lbm_launches + res["launches"]),
        }
        print(json.dumps(line))
    net.close()


def run_shear_track(args, rank, world, dist):
    """The 512 x 256 shear configuration run to its end for three solid-gas adsorption
    strengths: wetted width on the wall and detachment step, plus the throughput."""
    import torch
    from paper_2609_26332_b300 import shear
    betas = (0.0, 0.5, 1.0)
    t0 = time.perf_counter()
    res = shear.track(betas, steps=args.track_steps, every=500)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if rank == 0:
        cells = 512 * 256 * len(betas)
        line = {
            "metric": "sheared-drop contact-line tracking, wall-clock MLUPS", "value": cells * args.track_steps / dt / 1e6,
            "unit": "MLUPS", "n_gpus": world, "steps": args.track_steps, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "shear drop 512x256, R=60 at (128, 0), theta0=90, psi0=0.02, top wall 0.01, "
                                   "beta_sg in {0, 0.5, 1}, beta_sl=0, Ca=0.5 (sigma 0.002), Pi=1.35, Ex=0.5; "
                                   "three drops in one batch, wall row read every 500 steps"},
            "tracks": {str(b): {"detach_step": r["detach"], "width_first": r["width"][0], "width_last": r["width"][-1],
                                "centre_first": r["centre"][0], "centre_last": r["centre"][-1],
                                "width_every_5000": r["width"][9::10], "kinetic_final": r["kinetic"],
                                "range_count": r["range_count"]} for b, r in res.items()},
            "gpu_launches": args.track_steps,
        }
        print(json.dumps(line))


# the heaviest 3 x 3 convs of the warm-start network on 256 x 128 fields, batch 32:
# (level, Cin, Cout) of the decoder's first convs and one conv of each level
CONV_LAYERS = [(0, 96, 32), (1, 192, 64), (2, 256, 128), (0, 32, 32), (1, 64, 64), (2, 128, 128)]


def run_conv(args, rank, world, dist):
    """Convolutions of the warm-start network (3x3, NHWC, BF16 operands, FP32 accumulation on
    the tensor cores): forward, input gradient and weight gradient of each layer, batch 32 of
    256 x 128 fields.  Each launch is timed alone with CUDA events after a 256 MB write has
    flushed L2, so inputs come from HBM.  Roofline per op: the larger of FLOPs over the BF16
    tensor peak and algorithmic bytes over the HBM copy bandwidth; these layers have 20-90
    FLOP per byte, far below the ~270 of the ridge point, so HBM bounds every one of them."""
    import torch
    from paper_2609_26332_b300 import binding as B
    torch.manual_seed(rank)
    Bn, H0, W0 = 32, 128, 256
    rows = []
    st = torch.cuda.current_stream()
    launches = 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    hbm, hbm_kind = measured_peaks()
    tc, tc_kind = measured_bf16_peak()
    tot = {"us": 0.0, "bound_us": 0.0, "flop": 0.0, "bytes": 0.0}
    for lv, ci, co in CONV_LAYERS:
        H, W = H0 >> lv, W0 >> lv
        P = Bn * H * W
        x = torch.randn(Bn, H, W, ci, device="cuda").to(torch.bfloat16)
        w = (torch.randn(co, 3, 3, ci, device="cuda") * (2.0 / (9 * ci)) ** 0.5).to(torch.bfloat16)
        wt = torch.empty(ci, 3, 3, co, device="cuda", dtype=torch.bfloat16)
        y = torch.empty(Bn, H, W, co, device="cuda", dtype=torch.bfloat16)
        dx = torch.empty_like(x)
        dw = torch.zeros(co, 3, 3, ci, device="cuda", dtype=torch.float32)
        B.conv3x3_flip_weights(w, wt)
        flop = 2.0 * P * 9 * ci * co
        wbytes = 2.0 * 9 * ci * co
        # algorithmic bytes: operands read once, results written once
        ops = {"forward": (lambda: B.conv3x3_forward(x, w, None, y, relu=True), 2.0 * P * (ci + co) + wbytes),
               "input_grad": (lambda: B.conv3x3_input_grad(y, wt, x, dx), 2.0 * P * (co + 2 * ci) + wbytes),
               "weight_grad": (lambda: B.conv3x3_weight_grad(x, y, dw), 2.0 * P * (ci + co) + 2 * wbytes)}
        for name, (fn, nbytes) in ops.items():
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ms = 0.0
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            ms = ranks.max_over_ranks(ms / args.steps, dist, "cuda")
            launches += args.steps
            t_tc, t_mem = flop / (tc * 1e12) * 1e6, nbytes / (hbm * 1e9) * 1e6
            bound_us = max(t_tc, t_mem)
            rows.append({"layer": f"{H}x{W} {ci}->{co}", "op": name, "us": ms * 1e3, "tflops": flop / ms / 1e9,
                         "gbs": nbytes / ms / 1e6, "flop_per_byte": flop / nbytes,
                         "bound": "tensor" if t_tc > t_mem else "hbm", "frac": bound_us / (ms * 1e3)})
            tot["us"] += ms * 1e3
            tot["bound_us"] += bound_us
            tot["flop"] += flop
            tot["bytes"] += nbytes
        assert B.conv_error() == 0
    if rank == 0:
        achieved = tot["bytes"] / (tot["us"] * 1e-6) / 1e9
        print(json.dumps({
            "metric": "warm-start conv throughput (fwd + input grad + weight grad)",
            "value": world * tot["flop"] / (tot["us"] * 1e-6) / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot["us"] / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16-operands/f32-accumulate", "data": "synthetic",
            "config": {"workload": "3x3 convs of the warm-start network, batch 32 of 256x128 fields: "
                                   + ", ".join(f"level {lv} {ci}->{co}" for lv, ci, co in CONV_LAYERS),
                       "l2": "256 MB written before every timed launch"},
            # every op is HBM-bound (intensity below the ridge): the fraction is the sum of the
            # per-op roofline times over the sum of the measured times
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": tot["bound_us"] / tot["us"], "traffic": None, "peak_kind": hbm_kind,
                         "tensor_peak_tflops": tc, "tensor_peak_kind": tc_kind,
                         "tensor_frac": tot["flop"] / (tot["us"] * 1e-6) / 1e12 / tc},
            "layers": rows, "gpu_launches": launches,
        }))


# the three-dimensional step (D3Q19): 3 x 19 populations read and written plus 8 history
# values read and written, FP32
BYTES_PER_CELL_3D = 2 * (3 * 19 + 8) * 4


def run_3d(args, rank, world, dist):
    """The three-dimensional extension: a hemispherical surfactant drop on the bottom wall
    under a sliding top wall (the shear configuration's physics), nx x ny x nz =
    256 x 128 x 256 (8.4 M cells, the cell count of the 2D benchmark), three launches per
    step, CUDA events on the library's stream."""
    import torch
    from paper_2609_26332_b300 import binding as B, inputs
    nx, ny, nz = args.nx3, args.ny3, args.nz3
    cells = nx * ny * nz
    R = 0.375 * ny
    pb = inputs.bulk_phi(0.02, SHEAR_EX)
    phi0, psi0 = inputs.sessile_drop3d(nx, ny, nz, R, 4.0, phi_b=pb, psi0=0.02)
    stream = torch.cuda.current_stream()
    p = B.default_params(nx, ny, psi_b=0.02, sigma=SHEAR_SIGMA, Ex=SHEAR_EX, Pi=SHEAR_PI)
    d = B.Domain3D(p, nz, stream=stream)
    d.set_wall(0, 90.0, 0.5, 0.0, 0.0)
    d.set_wall(1, 90.0, 0.0, 0.0, 0.01)
    d.init_fields(phi0, psi0)
    d.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = ranks.max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    clocks = sampler.stop() if sampler else None
    tot = d.read_totals(check=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d.init_fields(phi0, psi0)
    d.step(args.steps)
    out = d.read_fields()
    e2e_s = ranks.max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    if rank == 0:
        peak, kind = measured_peaks()
        per_step = ms / 1e3 / args.steps
        achieved = BYTES_PER_CELL_3D * cells / per_step / 1e9
        print(json.dumps({
            "metric": "coupled-step MLUPS (3D)", "value": world * cells * args.steps / (ms / 1e3) / 1e6,
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"3D shear drop {nx}x{ny}x{nz} R={R:.0f} fp32 (D3Q19)", "cells": cells,
                       "parallelism": f"replicas{world}",
                       "l2": f"state {cells * 2 * (19 + 36 + 4 + 8 + 8) * 4 / 1e9:.2f} GB >> 126 MB L2, no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": kind, "bytes_per_cell": BYTES_PER_CELL_3D,
                         "kernels": ["moments3d", "potentials3d", "collide3d"]},
            "e2e": {"value": world * cells * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": 16 * cells / args.steps, "d2h_bytes_per_step": 48 * cells / args.steps},
            "gpu_launches": 3 * args.steps, "clocks": clocks,
            "totals": {"psi_total": tot["psi_total"], "lambda_phi": tot["lambda_phi"],
                       "range_count": tot["range_count"],
                       "phi_range": [float(out["phi"].min()), float(out["phi"].max())]},
        }))
    d.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--multiplier", default="paper", choices=["paper", "target", "exact"],
                    help="lambda_phi of the shear workload: Eq. eq15, its drift-correcting form, or the "
                         "exact root of the discrete constraint (one extra reduction pass per step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="shear", choices=["shear", "drop1000", "batch", "warmstart", "shear-track",
                                                             "conv", "3d"])
    ap.add_argument("--nx3", type=int, default=256)
    ap.add_argument("--ny3", type=int, default=128)
    ap.add_argument("--nz3", type=int, default=256)
    ap.add_argument("--track-steps", type=int, default=50000)
    ap.add_argument("--ws-train", type=int, default=4096)
    ap.add_argument("--ws-eval", type=int, default=256)
    ap.add_argument("--ws-epochs", type=int, default=600)
    ap.add_argument("--ws-batch", type=int, default=32)
    ap.add_argument("--ws-lr", type=float, default=2e-3)
    ap.add_argument("--ws-tol", type=float, default=1e-6)
    ap.add_argument("--ws-eval-tol", type=float, default=1e-6)
    ap.add_argument("--ws-max-steps", type=int, default=30000)
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--graph-steps", type=int, default=32)
    ap.add_argument("--tiling-cache", default=None)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = ranks.rank_world()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2609_26332_b300 import build as _build
    _build.build()
    from paper_2609_26332_b300 import binding as B
    if args.workload in ("batch", "warmstart", "shear-track", "conv", "3d"):
        {"batch": run_batch, "warmstart": run_warmstart, "shear-track": run_shear_track, "conv": run_conv,
         "3d": run_3d}[args.workload](
            args, rank, world, dist)
        if dist:
            dist.destroy_process_group()
        return

    case = (drop1000_case if args.workload == "drop1000" else shear_case)(args.nx, args.ny, args.precision)
    case["multiplier"] = args.multiplier
    exact = args.multiplier == "exact"
    cells = args.nx * args.ny
    stream = torch.cuda.current_stream()
    phi0, psi0 = init_fields(case)
    d = make_domain(case, stream)
    d.init_fields(phi0, psi0)
    d.step(args.warmup)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    ms_max = ranks.max_over_ranks(ms, dist, "cuda")
    tot = d.read_totals(check=False)

    # end to end through the C ABI with host buffers: upload, step, read back
    pin_phi = torch.from_numpy(phi0).pin_memory().numpy()
    pin_psi = torch.from_numpy(psi0).pin_memory().numpy()
    outs = {k: torch.empty((args.ny, args.nx), dtype=torch.float64).pin_memory().numpy()
            for k in ("phi", "psi", "ux", "uy", "p")}
    import ctypes
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    d.init_fields(pin_phi, pin_psi)
    d.step(args.steps)
    B.lib.slbm_read_fields(d._h, *[outs[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                   for k in ("phi", "psi", "ux", "uy", "p")])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = ranks.max_over_ranks(e2e_s, dist, "cuda")

    if rank == 0:
        peak, peak_kind = measured_peaks()
        per_launch_s = ms_max / 1e3 / args.steps
        # exact mode: both kernels of the step over the step time
        bpc = BYTES_PER_CELL[args.precision] + (EXACT_BYTES_PER_CELL[args.precision] if exact else 0)
        achieved = bpc * cells / per_launch_s / 1e9
        value = world * cells * args.steps / (ms_max / 1e3) / 1e6
        line = {
            "metric": "coupled-step MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": step_config(args, case, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": (TRAFFIC.get(kernel_hash(), {}).get(args.precision)
                                     if (args.nx, args.ny) == (4096, 2048) and not exact and args.workload == "shear"
                                     else None),
                         "peak_kind": peak_kind, "bytes_per_cell": bpc,
                         "kernels": ["step_kernel"] + (["exact_multiplier_kernel"] if exact else []),
                         "kernel_hash": kernel_hash()},
            "e2e": {"value": world * cells * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": 16 * cells / args.steps, "d2h_bytes_per_step": 40 * cells / args.steps},
            "gpu_launches": args.steps * (2 if exact else 1),
            "clocks": clocks,
            "totals": {"psi_total": tot["psi_total"], "lambda_phi": tot["lambda_phi"],
                       "range_count": tot["range_count"]},
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    d.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
