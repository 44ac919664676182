"""Learned warm start of sessile-drop relaxations (driver of the library's warm-start
entry points; every numerical step runs in libsurflbm.so).

* ``drop_specs``   seeded drop parameters: contact angle U[30, 150] deg, surfactant
                   load psi0 U[0.005, 0.05], adsorption strengths U[0, 1], initial
                   semicircle radius U[0.25, 0.35] ny
* ``cold_batch``   a batch of those drops on ny x nx grids, cold-started
* ``build_dataset`` relax cold starts to equilibrium with the batch solver and collect
                   the relaxed (phi, ln(psi / psi0)) fields on the device
* ``train``        Adam on the tensor-core network
* ``evaluate``     steps to equilibrium from cold and from warm starts of the same
                   drops, and the equilibrium contact angles of both
* ``contact_angle`` circle fit of the phi = 0 contour above the wall layer

The parameter rows handed to the network are (theta0 [deg], beta_sg, beta_sl, psi0,
area fraction), the area fraction being the initial semicircle's area / (nx ny).
"""
import math

import numpy as np

from . import binding as B
from . import inputs

EPS = 4.0


def drop_specs(count, seed, ny, nx):
    u = inputs.uniform(seed, 6 * count, stream=13).reshape(count, 6)
    out = []
    for k in range(count):
        out.append(dict(theta0=30.0 + 120.0 * u[k, 0], psi0=0.005 + 0.045 * u[k, 1], beta_sg=float(u[k, 2]),
                        beta_sl=float(u[k, 3]), R=(0.25 + 0.1 * u[k, 4]) * ny, ny=ny, nx=nx))
    return out


def cond_rows(specs):
    return np.array([[s["theta0"], s["beta_sg"], s["beta_sl"], s["psi0"],
                      0.5 * math.pi * s["R"] ** 2 / (s["nx"] * s["ny"])] for s in specs], dtype=np.float32)


def cold_fields(s):
    pb = inputs.bulk_phi(s["psi0"], 1.0)
    return inputs.sessile_drop(s["nx"], s["ny"], s["R"], EPS, phi_b=pb, psi0=s["psi0"])


def cold_batch(specs, stream=None, graph_steps=50, band_rows=128):
    params, walls = [], []
    for s in specs:
        params.append(B.default_params(s["nx"], s["ny"], psi_b=s["psi0"], multiplier=B.TARGET))
        walls.append(((s["theta0"], s["beta_sg"], s["beta_sl"], 0.0), (90.0, 0.0, 0.0, 0.0)))
    b = B.Batch(params, walls, stream=stream)
    for i, s in enumerate(specs):
        phi, psi = cold_fields(s)
        b.init_fields(i, phi, psi)
    b.set_tiling(band_rows, 2, graph_steps)
    return b


def build_dataset(net, specs, tol, max_steps, check_every=500, chunk=1024, stream=None, log=None):
    """Relax every spec from its cold start; returns (cond rows, device targets
    [S, 2, ny, nx] float32, steps) for the instances that converged, and the steps of
    all (-1: not converged, -2: diverged)."""
    import torch
    ny, nx = specs[0]["ny"], specs[0]["nx"]
    keep_cond, keep_t, all_steps = [], [], []
    launches = 0
    for c0 in range(0, len(specs), chunk):
        part = specs[c0:c0 + chunk]
        b = cold_batch(part, stream=stream)
        steps = b.run_to_equilibrium(tol, max_steps, check_every)
        all_steps.append(steps)
        launches += batch_steps_run(steps, max_steps)
        ok = np.nonzero(steps > 0)[0]
        t = torch.empty((len(ok), 2, ny, nx), dtype=torch.float32, device="cuda")
        for j, i in enumerate(ok):
            net.batch_targets(b, int(i), part[i]["psi0"], t[j])
        keep_t.append(t)
        keep_cond.append(cond_rows([part[i] for i in ok]))
        b.close()
        if log:
            log(f"dataset chunk {c0 // chunk}: {len(ok)}/{len(part)} converged, "
                f"{int((steps == -2).sum())} diverged, median steps {np.median(steps[ok]) if len(ok) else -1}")
    return np.concatenate(keep_cond), torch.cat(keep_t), np.concatenate(all_steps), launches


def batch_steps_run(steps, max_steps):
    """Time steps (one launch each) a run_to_equilibrium call took: max_steps if an
    instance never converged, else the step of the last convergence."""
    if (steps == -1).any():
        return int(max_steps)
    done = steps[steps > 0]
    return int(done.max()) if len(done) else 0


def train(net, cond, targets, epochs, batch_size, lr, seed=0, log=None, lr_final=None):
    """Minibatch Adam over the device dataset; cosine decay from lr to lr_final."""
    import torch
    S = cond.shape[0]
    cond_t = torch.tensor(cond, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    lr_final = lr * 0.05 if lr_final is None else lr_final
    steps_per_epoch = max(1, S // batch_size)
    total = epochs * steps_per_epoch
    hist = []
    k = 0
    for ep in range(epochs):
        perm = rng.permutation(S)
        acc = 0.0
        for j in range(steps_per_epoch):
            idx = torch.tensor(perm[j * batch_size:(j + 1) * batch_size], dtype=torch.int32, device="cuda")
            a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / total))
            acc += net.train_step(cond_t, targets, idx, a)
            k += 1
        hist.append(acc / steps_per_epoch)
        if log and (ep % 10 == 0 or ep == epochs - 1):
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def evaluate(net, specs, tol, max_steps, check_every=500, stream=None):
    """Steps to equilibrium from cold and warm starts of the same drops, and the
    equilibrium angles of both (NaN where a run did not converge)."""
    cold = cold_batch(specs, stream=stream)
    warm = cold_batch(specs, stream=stream)
    accepted = net.warm_start(warm, np.arange(len(specs)), cond_rows(specs))
    s_cold = cold.run_to_equilibrium(tol, max_steps, check_every)
    s_warm = warm.run_to_equilibrium(tol, max_steps, check_every)
    a_cold = np.full(len(specs), np.nan)
    a_warm = np.full(len(specs), np.nan)
    for i in range(len(specs)):
        if s_cold[i] > 0:
            a_cold[i] = contact_angle(cold.read_fields(i, which=("phi",))["phi"])
        if s_warm[i] > 0:
            a_warm[i] = contact_angle(warm.read_fields(i, which=("phi",))["phi"])
    cold.close()
    warm.close()
    return dict(steps_cold=s_cold, steps_warm=s_warm, angle_cold=a_cold, angle_warm=a_warm, accepted=accepted,
                launches=batch_steps_run(s_cold, max_steps) + batch_steps_run(s_warm, max_steps))


def contact_angle(phi, eps=EPS):
    """Equilibrium angle (deg) of a drop on the bottom wall: algebraic circle fit of the
    phi = 0 crossings (linear interpolation along grid lines) at heights above 2 eps;
    node (i, j) at (i, j + 1/2), wall at y = 0.  NaN if the fit is impossible."""
    ny, nx = phi.shape
    pts = []
    a, b = phi, np.roll(phi, -1, axis=1)
    js, is_ = np.nonzero((a > 0) != (b > 0))
    for j, i in zip(js, is_):
        pts.append((i + a[j, i] / (a[j, i] - b[j, i]), j + 0.5))
    a, b = phi[:-1], phi[1:]
    js, is_ = np.nonzero((a > 0) != (b > 0))
    for j, i in zip(js, is_):
        pts.append((float(i), j + 0.5 + a[j, i] / (a[j, i] - b[j, i])))
    pts = np.array([p for p in pts if p[1] > 2 * eps])
    if len(pts) < 6:
        return float("nan")
    x, y = pts[:, 0], pts[:, 1]
    xc0 = x.mean()
    x = (x - xc0 + nx / 2) % nx - nx / 2 + xc0      # unwrap around the mean (periodic x)
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    sol, *_ = np.linalg.lstsq(A, x * x + y * y, rcond=None)
    xc, yc = sol[0] / 2, sol[1] / 2
    R = math.sqrt(max(sol[2] + xc * xc + yc * yc, 0.0))
    if R <= 0:
        return float("nan")
    return math.degrees(math.acos(max(-1.0, min(1.0, -yc / R))))
