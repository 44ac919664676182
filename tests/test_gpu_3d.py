"""The three-dimensional extension (D3Q19, include/surflbm3d.h) on the GPU: element-wise
parity with the FP64 3D oracle, conservation to float-float rounding over long runs, and
the closed forms of a sphere and a sessile cap.

* parity after 100 steps on a hemispherical surfactant drop sitting on an adsorbing wall
  under a sliding top wall (both constraints; an odd-sized grid; nz = 1): phi, psi within
  1e-5, u within 1e-5 of its largest value plus an FP32 floor, p likewise;
* sum psi (and sum phi under the linear constraint) to 1e-12 over 3000 steps;
* a free sphere: lambda_phi = 2 sigma / R (Gibbs-Thomson, the 3D value of the appendix's
  sigma / R) within 3 % at R = 4 eps, at rest up to spurious currents;
* a sessile drop relaxes to a spherical cap whose contact angle is theta0 within 3 deg
  (Young's law through the wetting ghost closure of Eq. boundary).
"""
import math

import numpy as np
import pytest

from oracle import OracleParams, Wall, Oracle3D

pytestmark = pytest.mark.gpu


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(nx, ny, nz, R, eps=3.0, psi0=0.01, walls=((70.0, 0.2, 0.6, 0.0), (90.0, 0.0, 0.0, 0.004)),
          constraint="nonlinear", multiplier="paper", psi_on=True, sigma=0.01):
    from paper_2609_26332_b300 import binding as B, inputs
    phi, psi = inputs.sessile_drop3d(nx, ny, nz, R, eps, psi0=psi0, psi_noise=1e-4 if psi_on else 0.0)
    op = OracleParams(nx=nx, ny=ny, eps=eps, sigma=sigma, psi_b=psi0 if psi_on else 0.0, psi_on=psi_on,
                      constraint=constraint, multiplier=multiplier, walls=[Wall(*walls[0]), Wall(*walls[1])])
    o = Oracle3D(op, nz, phi, psi if psi_on else None)
    p = B.default_params(nx, ny, eps=eps, sigma=sigma, psi_b=psi0 if psi_on else 0.0, psi_on=1 if psi_on else 0,
                         constraint=B.LINEAR if constraint == "linear" else B.NONLINEAR,
                         multiplier=B.TARGET if multiplier == "target" else B.PAPER)
    d = B.Domain3D(p, nz)
    for w in (0, 1):
        d.set_wall(w, *walls[w])
    d.init_fields(phi, psi if psi_on else None)
    return o, d


CASES = {
    "hemisphere": dict(nx=20, ny=12, nz=16, R=6.0),
    "linear_target": dict(nx=20, ny=12, nz=16, R=6.0, constraint="linear", multiplier="target"),
    "odd_grid": dict(nx=13, ny=9, nz=7, R=4.0, walls=((120.0, 0.5, 0.0, 0.0), (60.0, 0.0, 0.3, -0.003))),
    "one_plane": dict(nx=24, ny=10, nz=1, R=6.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_3d_matches_the_oracle(name):
    _cuda()
    steps = 100
    o, d = _pair(**CASES[name])
    with d:
        o.step(steps)
        d.step(steps)
        fg, tg = d.read_fields(), d.read_totals()
    fo, to = o.fields(), o.totals()
    e = {k: float(np.abs(fg[k] - fo[k]).max()) for k in ("phi", "psi", "p")}
    umax = max(float(np.abs(fo[k]).max()) for k in ("ux", "uy", "uz"))
    pmax = float(np.abs(fo["p"]).max())
    e["u"] = max(float(np.abs(fg[k] - fo[k]).max()) for k in ("ux", "uy", "uz"))
    print(f"3D {name}: {e}, max|u| {umax:.2e}, max|p| {pmax:.2e}")
    assert e["phi"] < 1e-5 and e["psi"] < 1e-5
    # FP32 floor: the force is a difference of O(sigma / eps) potentials, ~1e-9 per step
    assert e["u"] < 1e-5 * umax + 2e-8
    assert e["p"] < 1e-5 * pmax + 2e-8
    assert abs(tg["psi_total"] - to["psi_total"]) <= 1e-12 * max(abs(to["psi_total"]), 1e-300)
    assert abs(tg["lambda_phi"] - to["lam"]) <= 1e-4 * abs(to["lam"]) + 1e-12
    assert tg["range_count"] == 0 and tg["clamp_count"] == 0


def test_3d_conserves_the_totals_over_long_runs():
    _cuda()
    for cons in ("nonlinear", "linear"):
        _, d = _pair(32, 20, 24, 8.0, constraint=cons)
        with d:
            t0 = d.read_totals()
            d.step(3000)
            t1 = d.read_totals()
        rel = abs(t1["psi_total"] - t0["psi_total"]) / t0["psi_total"]
        print(f"3D {cons}: sum psi drift {rel:.2e}, sum phi {t0['phi_total']:.6f} -> {t1['phi_total']:.6f}")
        assert rel < 1e-12
        if cons == "linear":
            assert abs(t1["phi_total"] - t0["phi_total"]) <= 1e-12 * abs(t0["phi_total"])


def test_3d_sphere_multiplier_is_twice_sigma_over_R():
    """Gibbs-Thomson in 3D: at rest mu_phi = lambda h'(phi) with lambda = 2 sigma / R."""
    _cuda()
    from paper_2609_26332_b300 import binding as B, inputs
    n, R, eps, sigma = 64, 16.0, 4.0, 0.01
    phi, _ = inputs.free_drop3d(n, n, n, R, eps)
    p = B.default_params(n, n, eps=eps, sigma=sigma, psi_on=0, psi_b=0.0, multiplier=B.TARGET)
    with B.Domain3D(p, n) as d:
        d.init_fields(phi)
        d.step(4000)
        f, t = d.read_fields(which=("phi", "ux", "uy", "uz")), d.read_totals()
    Rm = (3.0 * np.sum(0.5 * (f["phi"] + 1.0)) / (4 * np.pi)) ** (1.0 / 3.0)
    ratio = t["lambda_phi"] / (2 * sigma / Rm)
    umax = float(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2 + f["uz"] ** 2).max())
    print(f"3D sphere R {Rm:.3f}: lambda / (2 sigma / R) = {ratio:.4f}, max|u| {umax:.2e}")
    assert abs(ratio - 1.0) < 0.03
    assert umax < 1e-4        # spurious currents, 1e-3 of the capillary speed sigma / (rho nu)


def _cap_angle(phi):
    """Contact angle of a sessile drop from a least-squares sphere through the phi = 0
    crossings along the grid lines (points within two nodes of the wall left out)."""
    nz, ny, nx = phi.shape
    pts = []
    for ax in range(3):
        a = phi
        b = np.roll(phi, -1, axis=ax) if ax != 1 else np.concatenate([phi[:, 1:], phi[:, -1:]], axis=1)
        cz, cy, cx = np.nonzero((a > 0) != (b > 0))
        for z, y, x in zip(cz, cy, cx):
            t = a[z, y, x] / (a[z, y, x] - b[z, y, x])
            q = [float(x), y + 0.5, float(z)]
            q[(2, 1, 0)[ax]] += t          # array axes are (z, y, x)
            pts.append(q)
    P = np.array([q for q in pts if q[1] > 3.0])
    A = np.column_stack([P[:, 0], P[:, 1], P[:, 2], np.ones(len(P))])
    rhs = -(P ** 2).sum(axis=1)
    (D, E, F, G), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    c = -0.5 * np.array([D, E, F])
    Rs = math.sqrt(c @ c - G)
    return math.degrees(math.acos(max(-1.0, min(1.0, -c[1] / Rs)))), Rs


@pytest.mark.parametrize("theta0", [60.0, 120.0])
def test_3d_sessile_cap_reaches_young_angle(theta0):
    _cuda()
    from paper_2609_26332_b300 import binding as B, inputs
    nx, ny, nz, R, eps = 72, 36, 72, 14.0, 4.0
    phi, _ = inputs.sessile_drop3d(nx, ny, nz, R, eps)
    p = B.default_params(nx, ny, eps=eps, sigma=0.01, psi_on=0, psi_b=0.0, multiplier=B.TARGET)
    with B.Domain3D(p, nz) as d:
        d.set_wall(0, theta0)
        d.init_fields(phi)
        d.step(15000)
        f = d.read_fields(which=("phi",))
    theta, Rs = _cap_angle(f["phi"])
    print(f"3D sessile theta0 {theta0}: measured {theta:.2f} deg, sphere radius {Rs:.2f}")
    assert abs(theta - theta0) < 3.0
