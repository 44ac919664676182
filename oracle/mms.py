"""Manufactured-solution convergence harness of the scalar lattice Boltzmann equations
(test infrastructure only; Sec. 4.1, accuracy and mass conservation test).

The two Allen-Cahn equations of the model -- phi with its multiplier, psi with the
linear mass constraint -- are advanced by the oracle's scalar machinery (equilibria
``Oracle._scalar_eq``, the isotropic Laplacian, the source weighting R + dt/2 dR/dt by a
backward difference and the d(phi u)/dt correction of F_{i,2}) on a doubly periodic unit
square with a prescribed constant velocity, driven by the source terms that make

    phi^e = a e^{-t} sin 2pi(x - u_x t) cos 2pi(y - u_y t)          (a = 0.5)
    psi^e = 0.5 + 0.05 e^{-2t} cos 2pi(x - u_x t) sin 2pi(y - u_y t)

exact solutions (u = (0.05, -0.03), M = 0.01, beta = 0.03, kappa = 9.375e-6,
k_B T = 0.162, W = 0.24, lambda_s = 0; diffusive scaling dt = dx^2 / 0.15, the reading
of the printed time step that keeps the lattice velocity small).  Both multipliers are
the linear ones of this test: mean(mu_phi) and mean(mu_psi) of the discrete fields.

Units: lattice spacing and step 1; a physical rate r becomes r dt, a velocity u dt/dx,
a Laplacian nabla^2_lat / dx^2.  The part M kappa nabla^2 phi of -M mu_phi is carried by
the lattice diffusion, D_lat = M kappa dt / dx^2 = eta c_s^2 (tau - 1/2) at tau = 1; psi,
with lambda_s = 0, gets the same lattice diffusion and an explicit -D_lat nabla^2 psi in
its source, so that its net diffusion vanishes.

The exact error values of the paper's table depend on its unstated eta and rates:
parity of the values is unpinned; the harness checks the convergence order.  Much of the
error constant comes from the lattice's spreading of the source: the w_i R of a node
reaches its neighbours, so the applied source is R + (1/6) lap_lat R, a relative
O(8 pi^2 dx^2 / 6) error that the decaying phi^e (e^{-5} at t = 5) amplifies (adding the
source to the rest population alone gives 3x smaller E2_phi and 5x smaller E2_psi at
dx = 1/32, t = 1); it is second order like everything else.
"""
import math

import numpy as np

from .lattice import CS2, CX, CY, Q, W
from .lbm import Oracle, laplacian

U = (0.05, -0.03)
M, BETA, KAPPA, KT, WADS = 0.01, 0.03, 9.375e-6, 0.162, 0.24
AMP = 0.5

_CXf = CX.astype(np.float64)[:, None, None]
_CYf = CY.astype(np.float64)[:, None, None]
_Wf = W[:, None, None]


def exact(x, y, t):
    """(phi^e, psi^e) at physical time t on coordinate arrays x, y."""
    X = 2.0 * math.pi * (x - U[0] * t)
    Y = 2.0 * math.pi * (y - U[1] * t)
    return AMP * math.exp(-t) * np.sin(X) * np.cos(Y), 0.5 + 0.05 * math.exp(-2.0 * t) * np.cos(X) * np.sin(Y)


def mubar_psi_exact(t):
    """Spatial mean of mu_psi^e (printed closed form of Sec. 4.1, a = a_phi(t))."""
    a = AMP * math.exp(-t)
    return -BETA * (1.0 - a * a / 2.0 + 9.0 * a ** 4 / 64.0) + WADS * a * a / 8.0


def mu_phi_bulk(phi, psi):
    return 4.0 * BETA * (1.0 - psi) * (phi ** 3 - phi) + WADS * psi * phi


def mu_psi_bulk(phi, psi):
    return KT * np.log(psi / (1.0 - psi)) - BETA * (1.0 - phi ** 2) ** 2 + 0.5 * WADS * phi ** 2


def sources(x, y, t):
    """S_phi, S_psi (physical units) making (phi^e, psi^e) exact."""
    pe, qe = exact(x, y, t)
    lap_pe = -8.0 * math.pi ** 2 * pe                       # nabla^2 of sin(X) cos(Y)
    mu_phi_e = mu_phi_bulk(pe, qe) - KAPPA * lap_pe
    mu_psi_e = mu_psi_bulk(pe, qe)                           # lambda_s = 0
    s_phi = -pe + M * (mu_phi_e - 0.0)                       # mean of mu_phi^e is 0
    s_psi = -2.0 * (qe - 0.5) + M * (mu_psi_e - mubar_psi_exact(t))
    return s_phi, s_psi


def _periodic_pad(a):
    return np.pad(a, 1, mode="wrap")


def run(n, t_end=5.0, dt_factor=0.15):
    """(E2_phi, E2_psi, steps, drift_phi, drift_psi): relative L2 errors at t_end on an
    n x n grid, and the changes of sum phi (relative to sum |phi|) and of sum psi
    (relative to sum psi) over the run."""
    dx = 1.0 / n
    dt = dx * dx / dt_factor
    steps = int(round(t_end / dt))
    coords = np.arange(n) * dx
    x, y = np.meshgrid(coords, coords)
    ux, uy = U[0] * dt / dx, U[1] * dt / dx
    uxa, uya = np.full((n, n), ux), np.full((n, n), uy)
    D = M * KAPPA * dt / (dx * dx)                           # lattice diffusion of phi (and psi)
    eta = D / (CS2 * 0.5)                                    # tau = 1
    phi, psi = exact(x, y, 0.0)
    g = Oracle._scalar_eq(phi, uxa, uya, eta)
    h = Oracle._scalar_eq(psi, uxa, uya, eta)
    R_prev = None
    phiu_prev = None
    sum0 = (phi.sum(), np.abs(phi).sum(), psi.sum())
    for k in range(steps):
        t = k * dt
        phi, psi = g.sum(axis=0), h.sum(axis=0)
        lap_phi = laplacian(_periodic_pad(phi), n, n) / (dx * dx)
        lap_psi_lat = laplacian(_periodic_pad(psi), n, n)
        mu_phi = mu_phi_bulk(phi, psi) - KAPPA * lap_phi
        mu_psi = mu_psi_bulk(phi, psi)
        s_phi, s_psi = sources(x, y, t)
        # reaction terms with the linear multipliers; the -M kappa lap phi part of
        # -M mu_phi is the lattice diffusion, psi's lattice diffusion is cancelled
        R_phi = dt * (M * (-mu_phi_bulk(phi, psi) + mu_phi.mean()) + s_phi)
        R_psi = dt * (M * (-mu_psi + mu_psi.mean()) + s_psi) - D * lap_psi_lat
        phiu = np.stack([phi * ux, phi * uy])
        psiu = np.stack([psi * ux, psi * uy])
        if R_prev is None:                                   # first step: the backward differences start from zero
            R_prev = (R_phi, R_psi)
            phiu_prev = (phiu, psiu)
        geq = Oracle._scalar_eq(phi, uxa, uya, eta)
        heq = Oracle._scalar_eq(psi, uxa, uya, eta)
        out = []
        for pop, eq, R, Rp, fu, fup in ((g, geq, R_phi, R_prev[0], phiu, phiu_prev[0]),
                                        (h, heq, R_psi, R_prev[1], psiu, phiu_prev[1])):
            d = fu - fup
            srcA = _Wf * (_CXf * d[0] + _CYf * d[1]) / CS2
            post = pop - (pop - eq) + 0.5 * srcA + _Wf * (1.5 * R - 0.5 * Rp)   # BGK at s = 1
            new = np.empty_like(post)
            for q in range(Q):
                new[q] = np.roll(np.roll(post[q], CX[q], axis=1), CY[q], axis=0)
            out.append(new)
        g, h = out
        R_prev = (R_phi, R_psi)
        phiu_prev = (phiu, psiu)
    phi, psi = g.sum(axis=0), h.sum(axis=0)
    pe, qe = exact(x, y, steps * dt)
    e_phi = math.sqrt(float(np.sum((phi - pe) ** 2) / np.sum(pe ** 2)))
    e_psi = math.sqrt(float(np.sum((psi - qe) ** 2) / np.sum(qe ** 2)))
    return e_phi, e_psi, steps, abs(phi.sum() - sum0[0]) / sum0[1], abs(psi.sum() - sum0[2]) / sum0[2]


# ------------------------------------------------------------------ channel variant
# The same test on the channel geometry of the full step (x periodic, halfway walls at
# y = 0 and y = 1): the walls admit no normal velocity and a 90-degree neutral wall fixes
# zero normal gradients, so the prescribed velocity is (0.05, 0) and both manufactured
# fields vary as cos(2 pi y) across the channel:
#
#     phi^e = a e^{-t} sin 2pi(x - u_x t) cos 2pi y
#     psi^e = 0.5 + 0.05 e^{-2t} cos 2pi(x - u_x t) cos 2pi y
#
# The means of the potentials keep the closed forms above (sin^2, cos^2 average 1/2 and
# sin^4, cos^4 3/8 on the node sets used here; the logarithm is odd in cos X).  The run
# goes through the full Oracle (flow populations at the uniform velocity, walls sliding
# with it, no force on the flow, the nonlinear-free linear constraint), with the
# lattice parameters below.

U_CH = (0.05, 0.0)


def channel_exact(x, y, t):
    X = 2.0 * math.pi * (x - U_CH[0] * t)
    Y = 2.0 * math.pi * y
    a = AMP * math.exp(-t)
    return a * np.sin(X) * np.cos(Y), 0.5 + 0.05 * math.exp(-2.0 * t) * np.cos(X) * np.cos(Y)


def channel_sources(x, y, t):
    pe, qe = channel_exact(x, y, t)
    lap_pe = -8.0 * math.pi ** 2 * pe
    s_phi = -pe + M * (mu_phi_bulk(pe, qe) - KAPPA * lap_pe)
    s_psi = -2.0 * (qe - 0.5) + M * (mu_psi_bulk(pe, qe) - mubar_psi_exact(t))
    return s_phi, s_psi


def channel_setup(n, dt_factor=0.15):
    """OracleParams, node coordinates, dx, dt and the lattice velocity of the channel test
    on n x n nodes (node (i, j) at x = i dx, y = (j + 1/2) dx)."""
    from .params import OracleParams, Wall
    dx = 1.0 / n
    dt = dx * dx / dt_factor
    kappa_l = KAPPA / (dx * dx)                  # -kappa lap = -(kappa / dx^2) lap_lattice
    m_l = M * dt                                 # mobility per step
    D = m_l * kappa_l                            # lattice diffusion, = eta c_s^2 (tau - 1/2) at tau = 1
    u_l = U_CH[0] * dt / dx
    # sigma, eps from beta = 3 sigma / (4 eps), kappa = 3 eps sigma / 8; W = 4 beta / Ex;
    # k_B T = 4 beta Pi; M_phi kappa = eta c_s^2 (tau - 1/2) gives eta = 6 D; psi gets the same
    # lattice diffusion and M_0 = D cancels it (lambda_s = 0)
    p = OracleParams(nx=n, ny=n, tau_f=1.0, tau_g=1.0, tau_h=1.0,
                     sigma=math.sqrt(32.0 * BETA * kappa_l / 9.0), eps=math.sqrt(2.0 * kappa_l / BETA),
                     Ex=4.0 * BETA / WADS, Pi=KT / (4.0 * BETA), M_psi=m_l, eta_phi=6.0 * D, eta_psi=6.0 * D,
                     lambda_s=0.0, phi_b=1.0, constraint="linear", multiplier="paper",
                     walls=[Wall(90.0, 0.0, 0.0, u_l), Wall(90.0, 0.0, 0.0, u_l)])
    c = np.arange(n) * dx
    x, y = np.meshgrid(c, c + 0.5 * dx)
    return p, x, y, dx, dt, u_l


def run_channel(n, t_end=5.0):
    """(E2_phi, E2_psi, steps, drift_psi) of the channel test through the full Oracle."""
    p, x, y, dx, dt, u_l = channel_setup(n)
    steps = int(round(t_end / dt))
    phi0, psi0 = channel_exact(x, y, 0.0)

    def source(k):
        s_phi, s_psi = channel_sources(x, y, k * dt)
        return dt * s_phi, dt * s_psi

    o = Oracle(p, phi0, psi0, u0=(u_l, 0.0), source=source, force=False)
    sum0 = psi0.sum()
    o.step(steps)
    f = o.fields()
    pe, qe = channel_exact(x, y, steps * dt)
    e_phi = math.sqrt(float(np.sum((f["phi"] - pe) ** 2) / np.sum(pe ** 2)))
    e_psi = math.sqrt(float(np.sum((f["psi"] - qe) ** 2) / np.sum(qe ** 2)))
    return e_phi, e_psi, steps, abs(f["psi"].sum() - sum0) / sum0, f
