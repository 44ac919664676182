"""The benchmark workload itself against the oracle, element by element: the sheared drop
on 4096 x 2048 in FP32, stepped by the same launch configuration bench.py times (the
persistent grid of 2 CTAs per SM, each CTA marching ~440 rows across one or two strips,
staged through TMA boxes).  The oracle needs ~20 s and ~15 GB of host memory per step at
this size, so the comparison covers the first three steps (the first-step history rule
and two ordinary steps); smaller grids check long runs."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import bench
from oracle import Oracle, OracleParams, Wall


def test_bench_workload_first_steps_elementwise():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, ny, steps = 4096, 2048, 3
    case = bench.shear_case(nx, ny)
    phi0, psi0 = bench.init_fields(case)
    d = bench.make_domain(case, None)
    d.init_fields(phi0, psi0)
    d.step(steps)
    fg = d.read_fields()
    tg = d.read_totals()
    d.close()
    p = OracleParams(nx=nx, ny=ny, psi_b=case["psi0"], sigma=bench.SHEAR_SIGMA, Ex=bench.SHEAR_EX, Pi=bench.SHEAR_PI,
                     walls=[Wall(case["theta"], case["beta_sg"], case["beta_sl"], 0.0), Wall(90.0, 0, 0, case["u_w"])])
    o = Oracle(p, phi0, psi0)
    o.step(steps)
    fo = o.fields()
    to = o.totals()
    e = {k: float(np.abs(fg[k] - fo[k]).max()) for k in ("phi", "psi", "ux", "uy", "p")}
    scale = {k: float(np.abs(fo[k]).max()) for k in ("ux", "uy", "p")}
    print(f"4096x2048 shear, {steps} steps vs oracle: max abs errors {e}, field scales {scale}")
    assert e["phi"] < 1e-6 and e["psi"] < 1e-6
    # 1e-5 relative plus the FP32 floor of the velocity and pressure moments (2e-8; after
    # three steps u_y and p are themselves only ~1e-6 .. 1e-4)
    for k in ("ux", "uy", "p"):
        assert e[k] <= 1e-5 * scale[k] + 2e-8, k
    assert abs(tg["psi_total"] - to["psi_total"]) <= 1e-12 * to["psi_total"]
    assert tg["range_count"] == 0 and tg["clamp_count"] == 0
