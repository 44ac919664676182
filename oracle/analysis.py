"""Measurements on (phi, psi) fields used by the oracle pins (test infrastructure).

* ``contact_angle`` - circle fit of the phi = 0 contour of a sessile drop (Sec. 4.3,
  Eq. a: the equilibrium shape is the cap (x - x0)^2 + (y + R cos theta)^2 = R^2).
  Reading c16: crossings by linear interpolation along grid lines, points closer
  than ``skip`` to the wall dropped, algebraic (Kasa) least-squares circle fit,
  cos(theta) = -y_c / R_c with the wall at y = 0.
* ``zero_level_area`` - area of {phi > 0} from the triangle-split linear
  reconstruction of Sec. 4.1 (each grid cell split into two triangles, the phi = 0
  contour reconstructed linearly in each).

Node (i, j) sits at x = i, y = j + 1/2.
"""

import math
import numpy as np


def zero_crossings(phi, skip=0.0):
    """(x, y) points where linear interpolation between neighbouring nodes crosses 0."""
    ny, nx = phi.shape
    pts = []
    # horizontal grid lines (periodic in x)
    a = phi
    b = np.roll(phi, -1, axis=1)
    js, is_ = np.nonzero((a > 0) != (b > 0))
    for j, i in zip(js, is_):
        t = a[j, i] / (a[j, i] - b[j, i])
        pts.append((i + t, j + 0.5))
    # vertical grid lines
    a = phi[:-1]
    b = phi[1:]
    js, is_ = np.nonzero((a > 0) != (b > 0))
    for j, i in zip(js, is_):
        t = a[j, i] / (a[j, i] - b[j, i])
        pts.append((float(i), j + 0.5 + t))
    pts = [p for p in pts if p[1] > skip]
    return np.array(pts, dtype=np.float64).reshape(-1, 2)


def fit_circle(pts):
    """Kasa algebraic fit: minimise sum (x^2 + y^2 + D x + E y + F)^2."""
    x, y = pts[:, 0], pts[:, 1]
    A = np.column_stack([x, y, np.ones_like(x)])
    rhs = -(x * x + y * y)
    (D, E, F), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = -D / 2.0, -E / 2.0
    R = math.sqrt(xc * xc + yc * yc - F)
    return xc, yc, R


def unwrap_drop(phi):
    """Roll the field in x so that the liquid region does not straddle x = 0."""
    col = (phi > 0).any(axis=0)
    if not col.any():
        return phi, 0
    gaps = np.nonzero(~col)[0]
    if len(gaps) == 0:
        return phi, 0
    shift = -int(gaps[0])
    return np.roll(phi, shift, axis=1), shift


def contact_angle(phi, eps, skip=None):
    """Equilibrium contact angle (degrees) of the sessile drop touching the bottom wall."""
    skip = 2.0 * eps if skip is None else skip
    ph, _ = unwrap_drop(phi)
    pts = zero_crossings(ph, skip=skip)
    if len(pts) < 5:
        raise ValueError("too few contour points for a circle fit")
    xc, yc, R = fit_circle(pts)
    c = max(-1.0, min(1.0, -yc / R))
    return math.degrees(math.acos(c)), (xc, yc, R)


def _tri_fraction(v1, v2, v3):
    """Fraction of a triangle where the linear interpolant of the vertex values is > 0."""
    v = np.stack([v1, v2, v3])
    pos = (v > 0).sum(axis=0)
    out = np.zeros(v1.shape)
    out[pos == 3] = 1.0
    for npos in (1, 2):
        m = pos == npos
        if not m.any():
            continue
        vv = v[:, m]
        # the lone vertex is the one whose sign differs from the other two
        lone_pos = npos == 1
        lone = np.where(lone_pos, np.argmax(vv > 0, axis=0), np.argmax(vv <= 0, axis=0))
        idx = np.arange(vv.shape[1])
        a = vv[lone, idx]
        o1 = vv[(lone + 1) % 3, idx]
        o2 = vv[(lone + 2) % 3, idx]
        frac = (a * a) / ((a - o1) * (a - o2))
        out[m] = frac if lone_pos else 1.0 - frac
    return out


def zero_level_area(phi, periodic_x=True):
    """Area of {phi > 0} over the grid cells between nodes (Sec. 4.1 triangle split)."""
    a = phi[:-1]
    b = np.roll(phi, -1, axis=1)[:-1]
    c = phi[1:]
    d = np.roll(phi, -1, axis=1)[1:]
    if not periodic_x:
        a, b, c, d = a[:, :-1], b[:, :-1], c[:, :-1], d[:, :-1]
    # cell corners: a=(i,j), b=(i+1,j), c=(i,j+1), d=(i+1,j+1); split along a-d
    t1 = _tri_fraction(a, b, d)
    t2 = _tri_fraction(a, d, c)
    return float(0.5 * (t1.sum() + t2.sum()))
