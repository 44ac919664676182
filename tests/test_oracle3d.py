"""Pins of the three-dimensional oracle (D3Q19, Sec. 2.3 with d = 3, Sec. 3) against lattice
identities and textbook closed forms; nothing compares it with itself or with the GPU.

* D3Q19 moments to fourth order (the isotropy the Sec. 3 stencils and equilibria rely on);
* the isotropic gradient and Laplacian exact on quadratics in x, y and z;
* plane Couette flow between the walls exact (halfway bounce-back, moving wall);
* Fourier-mode diffusion along z at the rate D k^2, second order;
* a flat interface normal to z relaxes to tanh(2 z / eps), as in two dimensions;
* a surfactant drop on an adsorbing wall conserves sum psi to round-off;
* Young-Laplace for a sphere, 2 sigma / R, with the drop at rest; a planted sign slip in
  the z component of the force's gradient fails that pin.
"""
import math

import numpy as np
import pytest

from oracle import OracleParams, Wall
from oracle.lattice3d import CX, CY, CZ, W, OPP, MIRY, CS2, Q
from oracle import lbm3d
from oracle.lbm3d import Oracle3D, laplacian3, gradient3


def test_d3q19_isotropy():
    c = np.stack([CX, CY, CZ]).astype(float)
    assert Q == 19 and abs(W.sum() - 1.0) < 1e-15
    assert np.allclose(c @ W, 0.0, atol=1e-15)
    assert np.allclose((c * W) @ c.T, CS2 * np.eye(3), atol=1e-15)
    for a in range(3):
        for b in range(3):
            for cc in range(3):
                for d in range(3):
                    val = np.sum(W * c[a] * c[b] * c[cc] * c[d])
                    exp = CS2 ** 2 * ((a == b) * (cc == d) + (a == cc) * (b == d) + (a == d) * (b == cc))
                    assert abs(val - exp) < 1e-15
    for k in range(Q):
        assert (CX[OPP[k]], CY[OPP[k]], CZ[OPP[k]]) == (-CX[k], -CY[k], -CZ[k])
        assert (CX[MIRY[k]], CY[MIRY[k]], CZ[MIRY[k]]) == (CX[k], -CY[k], CZ[k])


def test_stencils_exact_on_quadratics():
    nz, ny, nx = 4, 5, 6
    zz, yy, xx = np.meshgrid(np.arange(-1, nz + 1), np.arange(-1, ny + 1) + 0.5, np.arange(-1, nx + 1), indexing="ij")
    x, y, z = xx.astype(float), yy, zz.astype(float)
    P = 0.3 - 1.1 * x + 0.7 * y + 0.2 * z + 0.25 * x * x - 0.4 * x * y + 0.9 * y * y + 0.6 * z * z \
        + 0.35 * x * z - 0.15 * y * z
    sh = (nz, ny, nx)
    xi, yi, zi = x[1:-1, 1:-1, 1:-1], y[1:-1, 1:-1, 1:-1], z[1:-1, 1:-1, 1:-1]
    lap = laplacian3(P, sh)
    assert np.allclose(lap, 2 * (0.25 + 0.9 + 0.6), atol=1e-12)
    gx, gy, gz = gradient3(P, sh)
    assert np.allclose(gx, -1.1 + 0.5 * xi - 0.4 * yi + 0.35 * zi, atol=1e-12)
    assert np.allclose(gy, 0.7 - 0.4 * xi + 1.8 * yi - 0.15 * zi, atol=1e-12)
    assert np.allclose(gz, 0.2 + 1.2 * zi + 0.35 * xi - 0.15 * yi, atol=1e-12)


def test_couette_linear_profile_exact():
    ny, U = 8, 0.01
    p = OracleParams(nx=3, ny=ny, psi_on=False, sigma=0.0, M_phi=0.0, walls=[Wall(90.0), Wall(90.0, u_x=U)])
    o = Oracle3D(p, 2, -np.ones((2, ny, 3)))
    o.step(3000)
    f = o.fields()
    y = np.arange(ny) + 0.5
    assert np.allclose(f["ux"], (U * y / ny)[None, :, None], rtol=0, atol=1e-12)
    assert np.abs(f["uy"]).max() < 1e-14 and np.abs(f["uz"]).max() < 1e-14


def test_diffusion_along_z_second_order():
    tau = 0.8
    D = (tau - 0.5) / 3.0
    errs = []
    for nz in (16, 32):
        p = OracleParams(nx=1, ny=2, psi_on=False, sigma=0.0, tau_g=tau, M_phi=0.0)
        z = np.arange(nz)
        phi0 = np.broadcast_to((0.01 * np.cos(2 * np.pi * z / nz))[:, None, None], (nz, 2, 1)).copy()
        o = Oracle3D(p, nz, phi0)
        o.step(30)
        a1 = np.abs(np.fft.rfft(o.fields()["phi"][:, 0, 0])[1])
        o.step(50)
        a2 = np.abs(np.fft.rfft(o.fields()["phi"][:, 0, 0])[1])
        rate = -math.log(a2 / a1) / 50
        k = 2 * np.pi / nz
        errs.append(abs(rate / (D * k * k) - 1.0))
    assert errs[1] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_flat_interface_normal_to_z_tanh_profile():
    """Sec. 2.2, Eq. eq_T1 in three dimensions: a flat interface normal to z relaxes to
    tanh(2 z / eps) with the same O(dx^2 / eps^2) lattice error as in 2D."""
    eps = 4.0
    nz = 64
    p = OracleParams(nx=1, ny=2, eps=eps, psi_on=False)
    z = np.arange(nz)
    prof = np.tanh(2 * (z - nz / 4) / eps) * np.tanh(2 * (3 * nz / 4 - z) / eps)
    o = Oracle3D(p, nz, np.broadcast_to(prof[:, None, None], (nz, 2, 1)).copy())
    o.step(1500)
    phi = o.fields()["phi"][:, 0, 0]
    i = np.nonzero((phi[:-1] < 0) & (phi[1:] >= 0))[0][0]
    z0 = i + phi[i] / (phi[i] - phi[i + 1])
    m = np.abs(z - z0) < 3 * eps
    err = np.abs(phi[m] - np.tanh(2 * (z[m] - z0) / eps)).max()
    assert err < 3e-2


def _sessile3d(nx=16, ny=10, nz=14, R=5.0, eps=3.0, theta=70.0, psi0=0.01, **kw):
    x = np.arange(nx)
    y = np.arange(ny) + 0.5
    z = np.arange(nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt((X - nx / 2) ** 2 + Y ** 2 + (Z - nz / 2) ** 2)
    phi = np.tanh(2 * (R - r) / eps)
    psi = np.full_like(phi, psi0)
    p = OracleParams(nx=nx, ny=ny, eps=eps, psi_b=psi0,
                     walls=[Wall(theta, 0.2, 0.6), Wall(90.0, 0.0, 0.0, 0.004)], **kw)
    return p, nz, phi, psi


def test_surfactant_conserved_to_round_off():
    p, nz, phi, psi = _sessile3d()
    o = Oracle3D(p, nz, phi, psi)
    s0 = o.totals()["psi_total"]
    o.step(60)
    s1 = o.totals()["psi_total"]
    assert abs(s1 - s0) <= 1e-13 * s0
    # the linear constraint conserves sum phi the same way
    p2, nz, phi, psi = _sessile3d(constraint="linear")
    o2 = Oracle3D(p2, nz, phi, psi)
    a0 = o2.totals()["phi_total"]
    o2.step(60)
    assert abs(o2.totals()["phi_total"] - a0) <= 1e-12 * abs(a0)


def _resting_sphere(steps):
    """A free drop at rest in the middle of the channel (neutral walls far from it), the
    target reading of Eq. eq15 holding its volume: lambda_phi and the pressure jump
    between its centre and the gas, each over 2 sigma / R_m (R_m the radius of the sphere
    of the same liquid volume), and the largest velocity."""
    nx = ny = nz = 24
    R, eps, sigma = 7.5, 2.5, 0.01
    x = np.arange(nx)
    y = np.arange(ny) + 0.5
    Z, Y, X = np.meshgrid(np.arange(nz), y, x, indexing="ij")
    r = np.sqrt((X - nx / 2) ** 2 + (Y - ny / 2) ** 2 + (Z - nz / 2) ** 2)
    phi = np.tanh(2 * (R - r) / eps)
    p = OracleParams(nx=nx, ny=ny, eps=eps, sigma=sigma, psi_on=False, multiplier="target")
    o = Oracle3D(p, nz, phi)
    o.step(steps)
    f = o.fields()
    dp = f["p"][nz // 2, ny // 2, nx // 2] - f["p"][0, 1, 0]
    Rm = (3.0 * np.sum(0.5 * (f["phi"] + 1.0)) / (4 * np.pi)) ** (1.0 / 3.0)
    umax = float(np.sqrt(f["ux"] ** 2 + f["uy"] ** 2 + f["uz"] ** 2).max())
    return o.log[-1]["lam"] / (2 * sigma / Rm), dp / (2 * sigma / Rm), umax


def test_laplace_jump_of_a_sphere():
    """Gibbs-Thomson and Young-Laplace in three dimensions: at equilibrium mu_phi =
    lambda h'(phi), the multiplier carries the mean curvature, lambda = 2 sigma / R (the
    2D value is sigma / R), and the potential-form force integrates across the interface
    to a pressure jump lambda (h(phi_b) - h(-phi_b)) = lambda.  At R = 3 eps with
    eps = 2.5 nodes: lambda within 8 %, the jump within 20 % (its lattice error is
    O(dx^2 / eps^2): 14 % here, 7 % at eps = 4, R = 12 in a longer run), spurious
    currents below 2e-4."""
    lam, jump, umax = _resting_sphere(600)
    print(f"3D sphere: lambda / (2 sigma / R) = {lam:.4f}, jump / (2 sigma / R) = {jump:.4f}, max|u| = {umax:.2e}")
    assert abs(lam - 1.0) < 0.08
    assert abs(jump - 1.0) < 0.20
    assert umax < 2e-4


def test_planted_z_force_slip_is_caught(monkeypatch):
    """A sign slip in the z component of the isotropic gradient (a plausible index
    mistake in the force) fails the resting-sphere pin."""
    orig = lbm3d.gradient3

    def bad(P, shape):
        gx, gy, gz = orig(P, shape)
        return gx, gy, -gz
    monkeypatch.setattr(lbm3d, "gradient3", bad)
    lam, jump, umax = _resting_sphere(600)
    print(f"planted slip: lambda ratio {lam:.4f}, jump ratio {jump:.4f}, max|u| {umax:.2e}")
    assert abs(lam - 1.0) >= 0.08 or abs(jump - 1.0) >= 0.20 or umax >= 2e-4
