"""Seeded synthetic initial fields for the droplet workloads.

This module is shared by the CUDA path and the FP64 oracle and holds none of the
method's arithmetic: it only draws reproducible random numbers and lays out
initial (phi, psi) fields of the shapes the paper's experiments use (sessile
semicircle, Sec. 4.3-4.5; ellipse, Sec. 4.1; several free drops, Sec. 4.2).  Node
(i, j) sits at x = i, y = j + 1/2; the bottom wall is y = 0.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) applied to a counter,
``u_i = splitmix64(key + i) >> 11 * 2^-53`` with ``key = splitmix64(seed ^ (stream << 40))``.
"""

import math
import numpy as np

DEFAULT_SEED = 20260926
_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, n, stream=0):
    """n uniform doubles in [0, 1) from the counter-based generator."""
    key = _splitmix64(np.array([np.uint64(seed) ^ (np.uint64(stream) << np.uint64(40))], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        z = _splitmix64(key + np.arange(n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def bulk_phi(psi_b, Ex):
    """Initial bulk value used to shape the initial profile: sqrt(1 - psi_b / (Ex (1 - psi_b)))."""
    if psi_b <= 0 or Ex <= 0:
        return 1.0
    return math.sqrt(1.0 - psi_b / (Ex * (1.0 - psi_b)))


def _coords(nx, ny):
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None] + 0.5
    return x, y


def sessile_drop(nx, ny, R, eps, xc=None, phi_b=1.0, psi0=0.0, psi_noise=0.0, seed=DEFAULT_SEED):
    """Semicircular drop of radius R centred on the bottom wall at (xc, 0):
    phi = phi_b tanh(2 phi_b (R - r) / eps); psi = psi0 + U(-psi_noise, psi_noise)."""
    if xc is None:
        xc = nx / 2.0
    x, y = _coords(nx, ny)
    r = np.sqrt((x - xc) ** 2 + y ** 2)
    phi = phi_b * np.tanh(2.0 * phi_b * (R - r) / eps)
    psi = np.full((ny, nx), float(psi0))
    if psi_noise > 0:
        psi = psi + psi_noise * (2.0 * uniform(seed, nx * ny).reshape(ny, nx) - 1.0)
    return phi, psi


def free_drop(nx, ny, R, eps, xc=None, yc=None, phi_b=1.0, psi0=0.0):
    """Circular drop away from the walls."""
    xc = nx / 2.0 if xc is None else xc
    yc = ny / 2.0 if yc is None else yc
    x, y = _coords(nx, ny)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return phi_b * np.tanh(2.0 * phi_b * (R - r) / eps), np.full((ny, nx), float(psi0))


def sessile_drop3d(nx, ny, nz, R, eps, xc=None, zc=None, phi_b=1.0, psi0=0.0, psi_noise=0.0, seed=DEFAULT_SEED):
    """Hemispherical drop of radius R centred on the bottom wall at (xc, 0, zc), arrays
    [z][y][x] (node (i, j, l) at x = i, y = j + 1/2, z = l): phi = phi_b tanh(2 phi_b (R - r)
    / eps); psi = psi0 + U(-psi_noise, psi_noise)."""
    xc = nx / 2.0 if xc is None else xc
    zc = nz / 2.0 if zc is None else zc
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None] + 0.5
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    r = np.sqrt((x - xc) ** 2 + y ** 2 + (z - zc) ** 2)
    phi = phi_b * np.tanh(2.0 * phi_b * (R - r) / eps)
    psi = np.full((nz, ny, nx), float(psi0))
    if psi_noise > 0:
        psi = psi + psi_noise * (2.0 * uniform(seed, nx * ny * nz).reshape(nz, ny, nx) - 1.0)
    return phi, psi


def free_drop3d(nx, ny, nz, R, eps, phi_b=1.0, psi0=0.0):
    """Spherical drop at the centre of the box, arrays [z][y][x]."""
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None] + 0.5
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 + (z - nz / 2.0) ** 2)
    return phi_b * np.tanh(2.0 * phi_b * (R - r) / eps), np.full((nz, ny, nx), float(psi0))


def ellipse(nx, ny, a, b, eps, phi_b=1.0):
    """Ellipse with semi-axes a (x) and b (y) centred in the box; the signed distance
    to the ellipse is approximated by the first-order formula F / |grad F| with
    F = sqrt((x/a)^2 + (y/b)^2) - 1 scaled by the local radius (zero level exact)."""
    x, y = _coords(nx, ny)
    X = x - nx / 2.0
    Y = y - ny / 2.0
    F = (X / a) ** 2 + (Y / b) ** 2 - 1.0
    gx, gy = 2 * X / a ** 2, 2 * Y / b ** 2
    d = -F / np.maximum(np.sqrt(gx * gx + gy * gy), 1e-12)
    return phi_b * np.tanh(2.0 * phi_b * d / eps)


def slab(nx, ny, x1, x2, eps, phi_b=1.0):
    """Liquid slab between two vertical interfaces x1 < x2 (flat-interface tests)."""
    x, _ = _coords(nx, ny)
    d = np.minimum(x - x1, x2 - x)
    phi = phi_b * np.tanh(2.0 * phi_b * d / eps)
    return np.repeat(phi, ny, axis=0)


def drop_field(nx, ny, n_drops, r_min, r_max, eps, min_gap, seed=DEFAULT_SEED, wall_gap=None, phi_b=1.0,
               max_tries=100000):
    """Several non-overlapping circular drops with radii U[r_min, r_max] and centres
    placed by seeded rejection sampling (gap >= min_gap between interfaces, and at
    least ``wall_gap`` from the walls).  Returns (phi, list of (xc, yc, R))."""
    wall_gap = min_gap if wall_gap is None else wall_gap
    u = uniform(seed, 3 * max_tries, stream=7)
    drops = []
    t = 0
    while len(drops) < n_drops:
        if t >= max_tries:
            raise RuntimeError("could not place the drops")
        R = r_min + (r_max - r_min) * u[3 * t]
        xc = nx * u[3 * t + 1]
        yc = wall_gap + R + (ny - 2 * (wall_gap + R)) * u[3 * t + 2]
        t += 1
        ok = True
        for (x2, y2, R2) in drops:
            dx = abs(xc - x2)
            dx = min(dx, nx - dx)
            if math.hypot(dx, yc - y2) < R + R2 + min_gap:
                ok = False
                break
        if ok:
            drops.append((xc, yc, R))
    x, y = _coords(nx, ny)
    d = np.full((ny, nx), -np.inf)
    for (xc, yc, R) in drops:
        dx = np.abs(x - xc)
        dx = np.minimum(dx, nx - dx)
        d = np.maximum(d, R - np.sqrt(dx ** 2 + (y - yc) ** 2))
    return phi_b * np.tanh(2.0 * phi_b * d / eps), drops


def batch_instances(count, seed=DEFAULT_SEED):
    """Parameters of the many-drop batch workload: nx in {64, 96, ..., 512}, ny = nx/2,
    theta0 ~ U[30, 150] deg, psi0 ~ U[0.005, 0.05], beta_sg, beta_sl ~ U[0, 1], R = 0.3 ny."""
    u = uniform(seed, 5 * count, stream=11).reshape(count, 5)
    sizes = np.arange(64, 513, 32)
    out = []
    for k in range(count):
        nx = int(sizes[min(int(u[k, 0] * len(sizes)), len(sizes) - 1)])
        ny = nx // 2
        out.append(dict(nx=nx, ny=ny, theta0=30.0 + 120.0 * u[k, 1], psi0=0.005 + 0.045 * u[k, 2],
                        beta_sg=float(u[k, 3]), beta_sl=float(u[k, 4]), R=0.3 * ny))
    return out
