"""Pins of the oracle's streaming, walls, flow collision and scalar diffusion against
textbook closed forms (single-phase channel flows, Fourier-mode diffusion)."""
import math

import numpy as np
import pytest

from oracle import Oracle, OracleParams, Wall


def _single_phase(nx, ny, **kw):
    """sigma = 0 switches every chemical-potential term off: the flow set alone."""
    walls = kw.pop("walls", [Wall(90.0), Wall(90.0)])
    p = OracleParams(nx=nx, ny=ny, psi_on=False, sigma=0.0, M_phi=0.0, walls=walls, **kw)
    return Oracle(p, -np.ones((ny, nx)))


@pytest.mark.parametrize("mrt", [(0.0, 0.0, 0.0, 0.0), (1.1, 1.3, 0.9, 0.0), (0.0, 0.0, 0.0, 1.6)])
def test_couette_linear_profile_exact(mrt):
    """Halfway bounce-back with the moving-wall term reproduces plane Couette flow
    u_x(y) = U y / H exactly (y = j + 1/2, H = ny) for any s0, s1, s3; a distinct
    fourth-order rate s4 only enters through the O(U^2) part of f^eq."""
    ny, U = 8, 0.01
    o = _single_phase(4, ny, walls=[Wall(90.0), Wall(90.0, u_x=U)], mrt_f=mrt)
    o.step(3000)
    f = o.fields()
    y = np.arange(ny) + 0.5
    tol = 1e-12 if mrt[3] == 0.0 else 1e-2 * U * U
    assert np.allclose(f["ux"], (U * y / ny)[:, None], rtol=0, atol=tol)
    assert np.abs(f["uy"]).max() < max(tol, 1e-14)


def test_poiseuille_exact_at_magic_relaxation():
    """With tau - 1/2 = sqrt(3/16) (Ginzburg's 'magic' TRT combination Lambda = 3/16,
    BGK being TRT with equal rates) halfway bounce-back gives the parabola
    u = G y (H - y) / (2 rho nu) exactly."""
    ny, G = 8, 1e-6
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    o = _single_phase(4, ny, tau_f=tau, Gx=G)
    o.step(2500)
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    exact = G * y * (ny - y) / (2 * nu)
    assert np.allclose(o.fields()["ux"], exact[:, None], rtol=1e-10, atol=0)


def test_poiseuille_second_order():
    """At tau = 0.8 the bounce-back error of the parabola is O(dx^2): halving dx
    divides the relative error by about 4."""
    errs = []
    for ny in (8, 16):
        G = 1e-6 * (8.0 / ny) ** 2
        o = _single_phase(4, ny, tau_f=0.8, Gx=G)
        o.step(9000 if ny == 16 else 2500)
        nu = 0.1
        y = np.arange(ny) + 0.5
        exact = G * y * (ny - y) / (2 * nu)
        errs.append(np.abs(o.fields()["ux"][:, 0] - exact).max() / exact.max())
    assert errs[1] < errs[0]
    assert 3.0 < errs[0] / errs[1] < 5.0


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_scalar_diffusion_rate_second_order(tau):
    """Pure diffusion of a Fourier mode (sigma = 0, u = 0): the decay rate per step
    tends to D k^2 with D = c_s^2 (tau - 1/2) (Sec. 3 relation M kappa = eta c_s^2 (1/s - 1/2));
    the relative error falls ~4x when the wavelength doubles.  With the specular
    scalar walls a y-uniform mode is untouched by the two walls."""
    D = (tau - 0.5) / 3.0
    errs = []
    for nx in (32, 64):
        p = OracleParams(nx=nx, ny=2, psi_on=False, sigma=0.0, tau_g=tau, M_phi=0.0)
        x = np.arange(nx)
        o = Oracle(p, np.repeat((0.01 * np.cos(2 * np.pi * x / nx))[None, :], 2, axis=0))
        o.step(40)
        a1 = np.abs(np.fft.rfft(o.fields()["phi"][0])[1])
        o.step(60)
        a2 = np.abs(np.fft.rfft(o.fields()["phi"][0])[1])
        rate = -math.log(a2 / a1) / 60
        k = 2 * np.pi / nx
        errs.append(abs(rate / (D * k * k) - 1.0))
    assert errs[1] < 1e-3
    if tau == 1.0:   # at tau = 1 the k^4 term of the lattice rate vanishes: higher order
        assert errs[0] / errs[1] > 10.0
    else:
        assert 3.0 < errs[0] / errs[1] < 5.0
