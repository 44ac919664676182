"""Pins of the oracle's lattice pieces against textbook facts and the paper's printed values.

Nothing here compares the oracle with itself: each check is a closed form, a
lattice identity, or a number printed in the paper (tests/golden).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.lattice import CX, CY, W, OPP, MIRY, CS2, moment_matrix, rate_vector
from oracle.lbm import laplacian, gradient, Oracle
from oracle.params import OracleParams, clean_solid_tensions, psi_c_of

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_values.json")


def test_d2q9_weights_isotropy():
    """D2Q9 moments up to fourth order (textbook): sum w = 1, sum w c = 0,
    sum w c_a c_b = cs^2 delta_ab, sum w c_a c_b c_c c_d = cs^4 (dd + dd + dd)."""
    c = np.stack([CX, CY]).astype(float)
    assert abs(W.sum() - 1.0) < 1e-15
    assert np.allclose(c @ W, 0.0, atol=1e-15)
    assert np.allclose((c * W) @ c.T, CS2 * np.eye(2), atol=1e-15)
    for a in range(2):
        for b in range(2):
            for cc in range(2):
                for d in range(2):
                    val = np.sum(W * c[a] * c[b] * c[cc] * c[d])
                    exp = CS2 ** 2 * ((a == b) * (cc == d) + (a == cc) * (b == d) + (a == d) * (b == cc))
                    assert abs(val - exp) < 1e-15
    for k in range(9):
        assert CX[OPP[k]] == -CX[k] and CY[OPP[k]] == -CY[k]
        assert CX[MIRY[k]] == CX[k] and CY[MIRY[k]] == -CY[k]


def test_mrt_inverse_and_equal_rate_limit():
    """M^-1 S M reduces to s I when every rate equals s (why MRT with equal rates is BGK)."""
    M = moment_matrix()
    Minv = np.linalg.inv(M)
    assert np.allclose(M @ Minv, np.eye(9), atol=1e-13)
    for s in (0.5, 1.25, 1.9):
        S = np.diag(rate_vector(s, s, s, s, s))
        assert np.allclose(Minv @ S @ M, s * np.eye(9), atol=1e-13)
    # natural moments of a single population are the monomials of its velocity
    for k in range(9):
        e = np.zeros(9)
        e[k] = 1.0
        cx, cy = CX[k], CY[k]
        assert np.allclose(M @ e, [1, cx, cy, cx * cx, cx * cy, cy * cy, cx * cx * cy, cx * cy * cy,
                                   cx * cx * cy * cy])


def test_collision_equal_rates_is_bgk():
    """The oracle's matrix collision with all rates s equals f - s (f - feq) + (1 - s/2) src."""
    rng = np.random.default_rng(3)
    p = OracleParams(nx=4, ny=3, psi_on=False, sigma=0.0)
    o = Oracle(p, np.zeros((3, 4)))
    f, feq, src = (rng.standard_normal((9, 3, 4)) for _ in range(3))
    s = np.full((9, 3, 4), 1.3)
    out = o._collide(f, feq, s, src)
    assert np.allclose(out, f - 1.3 * (f - feq) + (1 - 0.65) * src, atol=1e-13)


def _padded_poly(ny, nx, coef):
    a, b, c, d, e, f = coef
    jj, ii = np.meshgrid(np.arange(-1, ny + 1), np.arange(-1, nx + 1), indexing="ij")
    x = ii.astype(float)
    y = jj + 0.5
    return a + b * x + c * y + d * x * x + e * x * y + f * y * y, x[1:-1, 1:-1], y[1:-1, 1:-1]


def test_stencils_exact_on_quadratics():
    """The isotropic gradient and Laplacian (Sec. 3 stencils) are exact for quadratics."""
    ny, nx = 5, 6
    coef = (0.3, -1.1, 0.7, 0.25, -0.4, 0.9)
    P, x, y = _padded_poly(ny, nx, coef)
    a, b, c, d, e, f = coef
    assert np.allclose(laplacian(P, ny, nx), 2 * d + 2 * f, atol=1e-12)
    gx, gy = gradient(P, ny, nx)
    assert np.allclose(gx, b + 2 * d * x + e * y, atol=1e-12)
    assert np.allclose(gy, c + e * x + 2 * f * y, atol=1e-12)


def test_laplacian_fourier_symbol():
    """On cos(k x) the D2Q9 isotropic Laplacian returns 2 (cos k - 1) cos(k x)."""
    nx, ny = 16, 3
    k = 2 * np.pi * 3 / nx
    z = np.cos(k * np.arange(nx))[None, :].repeat(ny, axis=0)
    P = np.empty((ny + 2, nx + 2))
    P[1:-1, 1:-1] = z
    P[0, 1:-1] = z[0]
    P[-1, 1:-1] = z[0]
    P[:, 0] = P[:, -2]
    P[:, -1] = P[:, 1]
    assert np.allclose(laplacian(P, ny, nx), 2 * (np.cos(k) - 1) * z, atol=1e-13)


def test_paper_worked_values():
    """Sec. 4.4 prints sigma_sg0, sigma_sl0 for sigma = 0.0107 and psi_c = 0.017 for Ex = 1, Pi = 0.18407."""
    g = json.load(open(GOLDEN))
    t = g["clean_solid_tensions"]
    sg, sl = clean_solid_tensions(t["sigma"], t["theta0_deg"])
    assert abs(sg - t["sigma_sg0"]) < 5e-9
    assert abs(sl - t["sigma_sl0"]) < 5e-9
    lc = g["langmuir_constant"]
    assert abs(psi_c_of(lc["Ex"], lc["Pi"]) - lc["psi_c"]) < 5e-4


def test_constraint_function_identities():
    """Sec. 2.3: Q(u) = 2 h_phi(phi_b u) - 1 = 3u/2 - u^3/2 satisfies
    1 - Q(tanh z) = (1 - tanh z)^2 (2 + tanh z) / 2, and h_phi' integrates to 1 over
    [-phi_b, phi_b] (h(-phi_b) = 0, h(phi_b) = 1); checked on the oracle's g, g'."""
    g = json.load(open(GOLDEN))
    for phi_b in (1.0, 0.97):
        p = OracleParams(nx=2, ny=2, psi_on=False, phi_b=phi_b)
        o = Oracle(p, np.zeros((2, 2)))
        z = np.linspace(-3, 3, 41)
        t = np.tanh(z)
        Q = 2.0 * o._g(phi_b * t)
        assert np.allclose(1.0 - Q, 0.5 * (1 - t) ** 2 * (2 + t), atol=1e-14)
        xs = np.linspace(-phi_b, phi_b, 20001)
        integral = np.trapezoid(o._gprime(xs), xs)
        assert abs(integral - 1.0) < 1e-8
        assert abs(o._gprime(phi_b)) < 1e-15 and abs(o._gprime(-phi_b)) < 1e-15
    # c_0 = int sech^4 = 4/3 (appendix): the gradient energy of the tanh profile equals
    # sigma with kappa = 3 eps sigma / 8 and beta = 3 sigma / (4 eps)  (Sec. 2.1)
    eps, sigma = 4.0, 0.01
    beta, kappa = 3 * sigma / (4 * eps), 3 * eps * sigma / 8
    xx = np.linspace(-40, 40, 400001)
    ph = np.tanh(2 * xx / eps)
    dph = (2 / eps) / np.cosh(2 * xx / eps) ** 2
    tension = np.trapezoid(beta * (ph ** 2 - 1) ** 2 + 0.5 * kappa * dph ** 2, xx)
    assert abs(tension - sigma) < 1e-9
    assert abs(np.trapezoid(1 / np.cosh(xx) ** 4, xx) - g["tanh_identity"]["c0"]) < 1e-9
