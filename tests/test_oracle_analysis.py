"""Pins of the oracle's measurements on fields (Sec. 4.1 area, Sec. 4.3 contact angle)
against geometry with known answers: synthetic caps of given angle, circles and
ellipses of given area, and planes, for which the triangle-split linear reconstruction
is exact."""
import math

import numpy as np
import pytest

from oracle import analysis


def _cap(theta_deg, R=60.0, nx=260, ny=120, w=2.0, x0=130.0):
    """phi = tanh((R - r) / w) about (x0, -R cos theta): its zero contour is the circular
    cap meeting the wall y = 0 at the angle theta (nodes at x = i, y = j + 1/2).  The fit
    drops points within 2 eps of the wall, so the cap must rise well above that (a 45
    degree cap of radius 30 leaves less than a cell of arc there)."""
    y = np.arange(ny)[:, None] + 0.5
    x = np.arange(nx)[None, :]
    yc = -R * math.cos(math.radians(theta_deg))
    r = np.hypot(x - x0, y - yc)
    return np.tanh((R - r) / w)


@pytest.mark.parametrize("theta", [45.0, 90.0, 135.0])
def test_contact_angle_of_synthetic_caps(theta):
    th, (xc, yc, R) = analysis.contact_angle(_cap(theta), eps=4.0)
    assert abs(th - theta) < 0.3, th
    assert abs(R - 60.0) < 0.05 and abs(xc - 130.0) < 0.05


def test_a_flipped_centre_sign_is_caught(monkeypatch):
    """A plausible slip planted in the oracle -- the fitted centre's y taken with the
    wrong sign -- turns a 45 degree cap into a 135 degree one."""
    orig = analysis.fit_circle
    monkeypatch.setattr(analysis, "fit_circle", lambda pts: (lambda c: (c[0], -c[1], c[2]))(orig(pts)))
    th, _ = analysis.contact_angle(_cap(45.0), eps=4.0)
    assert abs(th - 45.0) > 10.0


def test_area_is_exact_for_planes():
    ny, nx = 40, 50
    j = np.arange(ny)[:, None].astype(float)
    i = np.arange(nx)[None, :].astype(float)
    j0, s = 13.37, 0.21
    phi = j - j0 - s * i                        # {phi > 0}: above the line j = j0 + s i
    W, H = nx - 1, ny - 1                       # the node rectangle [0, W] x [0, H]
    exact = W * (H - j0) - s * W * W / 2.0
    assert abs(analysis.zero_level_area(phi, periodic_x=False) - exact) < 1e-9


@pytest.mark.parametrize("a,b", [(20.0, 20.0), (28.0, 18.0)])
def test_area_of_circle_and_ellipse(a, b):
    ny, nx = 100, 120
    y = np.arange(ny)[:, None].astype(float)
    x = np.arange(nx)[None, :].astype(float)
    d = np.hypot((x - 60.3) / a, (y - 49.7) / b) - 1.0   # zero level set: the ellipse
    area = analysis.zero_level_area(-d)
    assert abs(area - math.pi * a * b) / (math.pi * a * b) < 2e-3
