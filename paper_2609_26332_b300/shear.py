"""Sheared sessile drop: Couette flow over the adsorbing wall, contact-line tracking and
detachment (driver of the library; every step runs in libsurflbm.so).

The drop (semicircle of radius R about (nx/4, 0), intrinsic angle theta0) sits on the
bottom wall; the top wall moves at u_w.  Parameters follow the paper's Couette case
(Sec. 4.5: Pi = 1.35, Ex = 0.5, Ca = mu u_w / sigma = 0.5, which with tau = 0.8 and
u_w = 0.01 gives sigma = 0.002) at the lattice sizes of the shear configuration.
Several adsorption strengths run as one batch; every `every` steps the phi = 0
crossings on the wall row give the wetted segments, and the drop counts as detached
at the first check with no wetted cell.
"""
import numpy as np

from . import binding as B
from . import inputs

SIGMA, EX, PI = 0.002, 0.5, 1.35


def shear_params(nx, ny, psi0=0.02, precision="fp32", **kw):
    return B.default_params(nx, ny, sigma=SIGMA, Ex=EX, Pi=PI, psi_b=psi0, precision=precision, **kw)


def initial_fields(nx, ny, R, psi0=0.02, eps=4.0):
    pb = inputs.bulk_phi(psi0, EX)
    return inputs.sessile_drop(nx, ny, R, eps, xc=nx / 4.0, phi_b=pb, psi0=psi0)


def wetted_segments(phi_row):
    """(left, right) x of every wetted (phi > 0) segment of a periodic wall row, with
    the ends at the linearly interpolated phi = 0 crossings (node i at x = i)."""
    n = len(phi_row)
    pos = phi_row > 0
    if pos.all():
        return [(0.0, float(n))]
    if not pos.any():
        return []
    segs = []
    start = int(np.argmin(pos))           # a dry node: walk the ring from there
    i = start
    for _ in range(n):
        j = (i + 1) % n
        if not pos[i] and pos[j]:
            a, b = phi_row[i], phi_row[j]
            left = i + a / (a - b)
        if pos[i] and not pos[j]:
            a, b = phi_row[i], phi_row[j]
            right = i + a / (a - b)
            if right < left:
                right += n
            segs.append((float(left), float(right)))
        i = j
    return segs


def track(betas_sg=(0.0, 0.5, 1.0), nx=512, ny=256, R=60.0, theta0=90.0, psi0=0.02, u_w=0.01, steps=50000,
          every=500, precision="fp32", stream=None):
    """Run one sheared drop per solid-gas adsorption strength (beta_sl = 0) as a batch.
    Returns per strength: check steps, wetted width, centre of the wetted region, the
    detachment step (None if still attached) and the final kinetic energy."""
    params = [shear_params(nx, ny, psi0, precision) for _ in betas_sg]
    walls = [((theta0, b, 0.0, 0.0), (90.0, 0.0, 0.0, u_w)) for b in betas_sg]
    phi0, psi_init = initial_fields(nx, ny, R, psi0)
    out = {b: dict(step=[], width=[], centre=[], detach=None) for b in betas_sg}
    with B.Batch(params, walls, stream=stream) as bt:
        for i in range(len(betas_sg)):
            bt.init_fields(i, phi0, psi_init)
        bt.set_tiling(64, 2, min(every, 250))
        done = 0
        while done < steps:
            n = min(every, steps - done)
            bt.step(n)
            done += n
            for i, b in enumerate(betas_sg):
                row = bt.read_fields(i, which=("phi",))["phi"][0]
                segs = wetted_segments(row)
                width = sum(r - l for l, r in segs)
                centre = float(np.mean([(l + r) / 2 for l, r in segs])) if segs else float("nan")
                out[b]["step"].append(done)
                out[b]["width"].append(width)
                out[b]["centre"].append(centre)
                if width == 0.0 and out[b]["detach"] is None:
                    out[b]["detach"] = done
        for i, b in enumerate(betas_sg):
            t = bt.read_totals(i, check=False)
            out[b]["kinetic"] = t["kinetic"]
            out[b]["range_count"] = t["range_count"]
    return out
