"""The manufactured-solution accuracy test of Sec. 4.1 run by the library's step kernel
(the channel form: x periodic, walls at y = 0 and 1; see ``slbm_set_mms``).

Physical test: M = 0.01, beta = 0.03, kappa = 9.375e-6, k_B T = 0.162, W = 0.24,
lambda_s = 0, amplitude 0.5, advection u = 0.05 along the channel, diffusive scaling
dt = dx^2 / 0.15.  ``lattice_params`` turns them into the library's lattice parameters
(unit spacing and step): kappa_l = kappa / dx^2 and M_l = M dt give sigma and eps through
beta = 3 sigma / (4 eps), kappa = 3 eps sigma / 8; W = 4 beta / Ex, k_B T = 4 beta Pi;
tau_g = tau_h = 1 with eta = 6 M_l kappa_l makes the lattice diffusion M_l kappa_l of phi
(and of psi, which M_0 = M_l kappa_l cancels, lambda_s = 0).
"""
import math

import numpy as np

from . import binding as B

PHYS = dict(amplitude=0.5, u=0.05, M=0.01, beta=0.03, kappa=9.375e-6, kT=0.162, W=0.24)


def grid(n):
    dx = 1.0 / n
    return dx, dx * dx / 0.15


def exact(n, t):
    """(phi^e, psi^e) at the nodes of the n x n channel at physical time t."""
    dx, _ = grid(n)
    x = np.arange(n) * dx
    y = (np.arange(n) + 0.5) * dx
    X = 2.0 * math.pi * (x[None, :] - PHYS["u"] * t)
    cY = np.cos(2.0 * math.pi * y)[:, None]
    phi = PHYS["amplitude"] * math.exp(-t) * np.sin(X) * cY
    psi = 0.5 + 0.05 * math.exp(-2.0 * t) * np.cos(X) * cY
    return phi, psi


def lattice_params(n):
    dx, dt = grid(n)
    kappa_l = PHYS["kappa"] / (dx * dx)
    m_l = PHYS["M"] * dt
    D = m_l * kappa_l
    beta = PHYS["beta"]
    p = B.default_params(n, n, tau_f=1.0, tau_g=1.0, tau_h=1.0,
                         sigma=math.sqrt(32.0 * beta * kappa_l / 9.0), eps=math.sqrt(2.0 * kappa_l / beta),
                         Ex=4.0 * beta / PHYS["W"], Pi=PHYS["kT"] / (4.0 * beta), M_psi=m_l,
                         eta_phi=6.0 * D, eta_psi=6.0 * D, lambda_s=0.0, phi_b=1.0, psi_b=0.5,
                         constraint=B.LINEAR, multiplier=B.PAPER)
    return p, PHYS["u"] * dt / dx


def run(n, t_end=5.0):
    """Relative L2 errors of phi and psi at t_end, the step count, the relative change of
    sum psi, and the fields."""
    dx, dt = grid(n)
    steps = int(round(t_end / dt))
    p, u_l = lattice_params(n)
    with B.Domain(p) as d:
        d.set_mms(dx=dx, dt=dt, **PHYS)
        for w in (0, 1):
            d.set_wall(w, 90.0, 0.0, 0.0, u_l)
        phi0, psi0 = exact(n, 0.0)
        d.init_fields(phi0, psi0)
        s0 = d.read_totals()["psi_total"]
        d.step(steps)
        f = d.read_fields()
        s1 = d.read_totals()["psi_total"]
    pe, qe = exact(n, steps * dt)
    e_phi = math.sqrt(float(np.sum((f["phi"] - pe) ** 2) / np.sum(pe ** 2)))
    e_psi = math.sqrt(float(np.sum((f["psi"] - qe) ** 2) / np.sum(qe ** 2)))
    return e_phi, e_psi, steps, abs(s1 - s0) / s0, f
