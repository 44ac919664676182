"""The benchmark's JSON contract, checked on the CPU through its reference arm (the FP64
oracle): one line with the required keys, the same workload config the GPU arm reports,
and, under a two-rank launch, a single line from rank 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    (j,) = _lines(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in j, k
    assert j["impl"] == "reference" and j["metric"] == "coupled-step MLUPS" and j["unit"] == "MLUPS"
    assert j["higher_is_better"] is True and j["steps"] == 2 and j["warmup"] >= 3 and j["value"] > 0
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    assert j["e2e"]["value"] == j["value"] and j["cpu_baseline"]["value"] == j["value"]
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    # the GPU arm's default config (same builder, same arguments)
    import argparse
    import bench
    args = argparse.Namespace(nx=4096, ny=2048, precision="fp32", workload="shear", multiplier="paper")
    assert j["config"] == bench.step_config(args, bench.shear_case(4096, 2048), 1)


def test_reference_arm_prints_once_under_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    (j,) = _lines(r.stdout)
    assert j["n_gpus"] == 2


def test_kernel_hash_ignores_comments_and_layout():
    import bench
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* no overflow\n check */ }\n"
    b = "int f(int x) { return 2 * x; }"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only("return 2 * x;") != bench.code_only("return 3 * x;")
    assert bench.state_bytes_per_cell("fp32") == 264 and bench.state_bytes_per_cell("bf16") == 152


def test_clock_sampler_reads_nvml_reasons(monkeypatch):
    """The clock record of the timed region from a fake NVML (reads only): median SM clock,
    the device's maximum, and the throttle reasons seen in any sample by name."""
    import types
    import time
    import bench
    fake = types.SimpleNamespace(NVML_CLOCK_SM=0, nvmlClocksEventReasonHwSlowdown=0x8,
                                 nvmlClocksEventReasonHwThermalSlowdown=0x40,
                                 nvmlClocksEventReasonSwThermalSlowdown=0x20, nvmlClocksEventReasonSwPowerCap=0x4)
    clocks = iter([1900.0, 2032.0, 2032.0] + [2032.0] * 10000)
    masks = iter([0x0, 0x4, 0x1] + [0x0] * 10000)
    fake.nvmlInit = lambda: None
    fake.nvmlDeviceGetHandleByPciBusId = lambda bus: "h"
    fake.nvmlDeviceGetHandleByIndex = lambda i: "h"
    fake.nvmlDeviceGetMaxClockInfo = lambda h, kind: 2032
    fake.nvmlDeviceGetClockInfo = lambda h, kind: next(clocks)
    fake.nvmlDeviceGetCurrentClocksEventReasons = lambda h: next(masks)
    monkeypatch.setitem(sys.modules, "pynvml", fake)
    s = bench.ClockSampler(0, period_s=0.001)
    time.sleep(0.02)
    rec = s.stop()
    assert rec["source"].startswith("nvml") and rec["samples"] >= 3
    assert rec["sm_max_mhz"] == 2032 and rec["sm_mhz"] == 2032.0
    assert rec["reasons"] == ["sw_power_cap"]   # 0x1 (idle) is not a throttle reason
