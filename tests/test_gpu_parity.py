"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element, on seeded inputs.  Tolerances: 1e-5 max-abs on phi and psi; on u and p 1e-5
relative to the oracle's max |u|, max |p|, plus an FP32 floor of 2e-8 absolute (u and p
are moments of FP32 populations of size up to ~1e-2, whose rounding, ~1e-9 per value and
step, leaves ~1e-8 after a few hundred steps; measured 5e-9 .. 1e-8 on every case);
conserved totals to 1e-12 relative."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import CONFIG1, make_case, oracle_for, domain_for


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _compare(c, steps=None, tol_phi=1e-5, tol_u=1e-5, precision="fp32"):
    _cuda()
    steps = c["steps"] if steps is None else steps
    o = oracle_for(c)
    o.step(steps)
    fo = o.fields()
    to = o.totals()
    with domain_for(c, precision=precision) as d:
        d.step(steps)
        fg = d.read_fields()
        tg = d.read_totals()
    umax = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max(), 1e-30)
    pmax = max(np.abs(fo["p"]).max(), 1e-30)
    du = max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max())
    dp = np.abs(fg["p"] - fo["p"]).max()
    err = {
        "phi": np.abs(fg["phi"] - fo["phi"]).max(),
        "psi": np.abs(fg["psi"] - fo["psi"]).max(),
        "u": du / umax,
        "p": dp / pmax,
        # within the stated bound: 1e-5 relative plus the FP32 floor
        "u_ok": du <= 1e-5 * umax + U_FLOOR,
        "p_ok": dp <= 1e-5 * pmax + U_FLOOR,
    }
    return err, fo, fg, to, tg


U_FLOOR = 2e-8


def test_config1_1000_steps():
    err, fo, fg, to, tg = _compare(CONFIG1)
    print("config1 errors", err)
    assert err["phi"] < 1e-5
    assert err["psi"] < 1e-5
    assert err["u"] < 1e-5            # max |u| is 1.3e-3 here: well above the floor
    assert err["p_ok"]
    assert abs(tg["psi_total"] - to["psi_total"]) / to["psi_total"] < 1e-12
    assert tg["clamp_count"] == 0 and tg["range_count"] == 0
    assert abs(tg["lambda_phi"] - to["lam"]) < 1e-4 * abs(to["lam"])


CASES = [
    make_case("ragged_small", 45, 19, 60, walls=((70.0, 0.3, 0.6, 0.0), (110.0, 0.5, 0.1, 0.0)), R=7.0),
    make_case("moving_wall", 70, 33, 120, walls=((90.0, 0.5, 0.0, 0.0), (90.0, 0.0, 0.0, 0.01)), R=10.0,
              psi0=0.02),
    make_case("linear_target", 64, 40, 100, walls=((120.0, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=12.0,
              constraint="linear", multiplier="target"),
    make_case("nonlinear_target", 64, 40, 100, walls=((50.0, 0.0, 0.9, 0.0), (90.0, 0.0, 0.0, 0.0)), R=12.0,
              multiplier="target"),
    make_case("clean", 80, 36, 100, walls=((45.0, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=12.0, psi_on=False),
    make_case("mrt", 48, 34, 80, walls=((75.0, 0.2, 0.4, 0.0), (90.0, 0.0, 0.0, 0.005)), R=10.0,
              mrt_f=(1.0, 1.1, 1.2, 1.3), mrt_g=(1.0, 1.4, 0.9, 1.1), mrt_h=(1.0, 1.5, 1.2, 1.0)),
    make_case("density_ratio", 64, 36, 80, walls=((80.0, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=10.0,
              rho_l=2.0, rho_g=1.0, tau_f_gas=0.7, Gy=-1e-6),
    make_case("free_drops", 96, 64, 80, init="drops", n_drops=3, psi0=0.015),
]


@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_parity_cases(c):
    err, fo, fg, to, tg = _compare(c)
    print(c["name"], err)
    assert err["phi"] < 1e-5
    assert err["psi"] < 1e-5
    assert err["u_ok"] and err["p_ok"]
    if c["psi_on"]:
        assert abs(tg["psi_total"] - to["psi_total"]) / to["psi_total"] < 1e-12


def test_first_step_and_zero_steps():
    """Fields at step 0 are the initial fields; one step matches element-wise."""
    c = make_case("tiny", 33, 17, 1, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=6.0)
    err0, fo, fg, _, _ = _compare(c, steps=0)
    # the first pull is exact up to the 2^-30 fixed-point grid of the exchanged populations
    assert err0["phi"] < 1e-7 and err0["psi"] < 1e-7
    err1, *_ = _compare(c, steps=1)
    assert err1["phi"] < 1e-6 and err1["psi"] < 1e-6 and err1["u_ok"] and err1["p_ok"]


def test_surfactant_conservation_gpu():
    """sum psi stays at its initial value to 1e-12 relative over 2000 steps (FP32 storage)."""
    _cuda()
    with domain_for(CONFIG1) as d:
        t0 = d.read_totals()
        for _ in range(4):
            d.step(500)
            t = d.read_totals()
            assert abs(t["psi_total"] - t0["psi_total"]) / t0["psi_total"] < 1e-12


@pytest.mark.parametrize("nx,ny,R", [(1, 24, 8.0), (5, 2, 1.5), (2, 3, 1.0)])
def test_degenerate_grids(nx, ny, R):
    """One periodic column (every x neighbour is the node itself), and channels of two and
    three rows (every row a wall row, the ghost and mirror rules meeting): element-wise
    against the oracle after 50 steps, sum psi to 1e-12."""
    c = make_case(f"deg_{nx}x{ny}", nx, ny, 50, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=R)
    err, fo, fg, to, tg = _compare(c)
    print(c["name"], err)
    assert err["phi"] < 1e-5 and err["psi"] < 1e-5
    # velocities here are a small transient (6e-5 in the column): besides 1e-4 relative,
    # allow the FP32 rounding of the force (|mu| ~ 3e-3, ~2e-10 per step) over 50 steps
    umax = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max())
    assert err["u"] * umax < 1e-4 * umax + 2e-8
    assert abs(tg["psi_total"] - to["psi_total"]) / to["psi_total"] < 1e-12
