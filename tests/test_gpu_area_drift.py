"""Geometric-area preservation of a relaxing elliptical drop (Sec. 4.1, Fig. 1): the
nonlinear constraint, imposed exactly on the lattice field (exact multiplier), against
the classical linear constraint.  The area of {phi > 0} is measured by the triangle-split
linear reconstruction of Sec. 4.1.  The linear constraint loses area at first order in
eps (its bulk shift); the nonlinear one keeps it to a level set by the area measurement
itself at 256^2 (about 6e-5: the piecewise-linear reconstruction errs differently on the
initial ellipse and on the relaxed circle, independently of eps).  On the paper's 1024^2
grid with eps = 18 .. 30 cells that floor is 16x lower (measured: 3.9e-6 .. 5.2e-6 over
eps = 18 .. 30, the eps-dependent part at most 1.3e-6, too close to the floor to fit an
order)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle.analysis import zero_level_area


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ellipse(n, eps):
    a, b = 0.28 * n, 0.18 * n
    y = np.arange(n)[:, None] + 0.5
    x = np.arange(n)[None, :] + 0.0
    X, Y = x - n / 2, y - n / 2
    r, th = np.hypot(X, Y), np.arctan2(Y, X)
    Rth = a * b / np.sqrt((b * np.cos(th)) ** 2 + (a * np.sin(th)) ** 2)
    return np.tanh(2.0 * (Rth - r) / eps)      # zero level set: the ellipse (a, b)


def _area_drift(n, eps, steps, linear):
    from paper_2609_26332_b300 import binding as B
    phi0 = _ellipse(n, eps)
    p = B.default_params(n, n, eps=eps, psi_on=0, constraint=B.LINEAR if linear else B.NONLINEAR,
                         multiplier=B.PAPER if linear else B.EXACT)
    with B.Domain(p) as d:
        d.set_wall(0, 90.0)
        d.set_wall(1, 90.0)
        d.init_fields(phi0)
        d.step(steps)
        phi = d.read_fields(("phi",))["phi"]
    A0 = zero_level_area(phi0)
    return abs(zero_level_area(phi) - A0) / A0


def test_nonlinear_constraint_preserves_area_far_better_than_linear():
    _cuda()
    epss = [4.0, 5.0, 6.0, 7.0, 8.0]
    lin = np.array([_area_drift(256, e, 20000, True) for e in epss])
    non = np.array([_area_drift(256, e, 20000, False) for e in epss])
    slope_lin = np.polyfit(np.log(epss), np.log(lin), 1)[0]
    print("256^2 linear E", lin, "slope", slope_lin, "nonlinear E", non)
    assert 0.8 < slope_lin < 1.1 and lin.min() > 1e-2
    assert non.max() < 2e-4 and (non < lin / 50).all()


def test_area_drift_on_the_papers_grid():
    _cuda()
    epss = [18.0, 21.0, 24.0, 27.0, 30.0]
    non = np.array([_area_drift(1024, e, 60000, False) for e in epss])
    slope = np.polyfit(np.log(epss), np.log(non), 1)[0]
    print("1024^2 nonlinear E", non, "slope", slope)
    assert non.max() < 2e-5 and non.min() < 6.25e-5 / 8
