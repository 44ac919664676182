"""The coupled lattice Boltzmann step in three dimensions, numpy float64 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.3 states the model for d = 2 and 3, and Sec. 3 writes its lattice Boltzmann
scheme for a general DdQq lattice; the paper's runs are all two-dimensional.  This is
the same scheme on D3Q19 for all three sets (flow f, phase field g, surfactant h), with
the single-relaxation-time collision (the MRT of Sec. 3 with all rates of a set equal,
which is what every configuration here uses), on a channel: x and z periodic, solid
walls half a spacing below row y = 0 and above row y = ny - 1.  Arrays are [z][y][x]
(node (i, j, l) at x = i, y = j + 1/2, z = l).

Each step, in the paper's order (the same as the two-dimensional oracle):
1.  phi = sum g, psi = sum h;
2.  wall ghost planes phi_G, psi_G from Eq. boundary (the same ghost closure as in 2D:
    phi_G = phi_0 - (df_w/dphi)/kappa, psi_G = psi_0 - (df_w/dpsi)/lambda_s);
3.  mu_phi, mu_psi (Eqs. eq_muphi, eq_mupsi) with the isotropic D3Q19 Laplacian
    sum_i 2 w_i [z(x + c_i) - z(x)] / c_s^2;
4.  lambda_phi = sum h' mu / sum h'^2 (Eq. eq15; or the target reading), mubar_psi =
    mean mu_psi (Eq. AC_psi);
5.  F = -phi grad mu_phi - psi grad mu_psi + G (Eq. eq_Fs0) with the isotropic gradient
    sum_i w_i c_i z(x + c_i) / c_s^2, rho u = sum c_i f_i + F/2, the pressure of Sec. 3;
6.  equilibria, the sources F_{i,1}, F_{i,2}, F_{i,3} of Sec. 3 and the BGK collision
    f* = f - s (f - f^eq) + (1 - s/2) F_i (+ w_i (1.5 R^n - 0.5 R^{n-1}) for the scalars);
7.  pull streaming: halfway bounce-back with the moving-wall term for f (wall speed along
    x), specular reflection for g and h, x and z periodic.
"""

import numpy as np

from .lattice3d import CX, CY, CZ, W, OPP, MIRY, CS2, Q
from .lbm import Oracle
from .params import derive

_CXf = CX.astype(np.float64)[:, None, None, None]
_CYf = CY.astype(np.float64)[:, None, None, None]
_CZf = CZ.astype(np.float64)[:, None, None, None]
_Wf = W[:, None, None, None]


def pad3(a, bottom, top):
    """[z][y][x] array padded by one node on every side: ghost planes below row y = 0
    (bottom) and above row y = ny - 1 (top), periodic images in x and z."""
    nz, ny, nx = a.shape
    P = np.empty((nz + 2, ny + 2, nx + 2))
    P[1:-1, 1:-1, 1:-1] = a
    P[1:-1, 0, 1:-1] = bottom
    P[1:-1, -1, 1:-1] = top
    P[:, :, 0] = P[:, :, -2]
    P[:, :, -1] = P[:, :, 1]
    P[0] = P[-2]
    P[-1] = P[1]
    return P


def neighbor3(P, k, shape):
    """Value at x + c_k from a padded array."""
    nz, ny, nx = shape
    return P[1 + CZ[k]:1 + CZ[k] + nz, 1 + CY[k]:1 + CY[k] + ny, 1 + CX[k]:1 + CX[k] + nx]


def laplacian3(P, shape):
    """Isotropic Laplacian on D3Q19 (Sec. 3 stencil form)."""
    c = P[1:-1, 1:-1, 1:-1]
    out = np.zeros(shape)
    for k in range(1, Q):
        out += W[k] * (neighbor3(P, k, shape) - c)
    return 2.0 * out / CS2


def gradient3(P, shape):
    """Isotropic gradient on D3Q19 (Sec. 3 stencil form)."""
    g = [np.zeros(shape), np.zeros(shape), np.zeros(shape)]
    for k in range(1, Q):
        nb = neighbor3(P, k, shape)
        g[0] += W[k] * CX[k] * nb
        g[1] += W[k] * CY[k] * nb
        g[2] += W[k] * CZ[k] * nb
    return g[0] / CS2, g[1] / CS2, g[2] / CS2


class Oracle3D(Oracle):
    """Plain FP64 three-dimensional implementation (D3Q19, BGK) of the coupled step.
    ``params`` is an OracleParams whose nx, ny are the x and y sizes; nz is the third.
    The wall formulas (Eqs. boundary, fw0, langmuir and the Remark-1 cap) and the
    constraint functions are those of the two-dimensional oracle (inherited helpers,
    evaluated plane by plane); the multiplier modes are "paper" and "target"."""

    def __init__(self, params, nz, phi0, psi0=None):
        p = params
        if p.multiplier not in ("paper", "target"):
            raise ValueError("the 3D oracle has the paper and target multipliers")
        if any(v != 0 for v in tuple(p.mrt_f) + tuple(p.mrt_g) + tuple(p.mrt_h)):
            raise ValueError("the 3D oracle collides with a single relaxation time")
        self.p = p
        self.source = None
        self.force = True
        self.d = derive(p)
        self.nz, self.ny, self.nx = int(nz), p.ny, p.nx
        self.shape = (self.nz, self.ny, self.nx)
        phi0 = np.asarray(phi0, dtype=np.float64)
        if phi0.shape != self.shape:
            raise ValueError("phi0 must be (nz, ny, nx)")
        psi0 = np.zeros_like(phi0) if (psi0 is None or not p.psi_on) else np.asarray(psi0, dtype=np.float64)
        z = np.zeros_like(phi0)
        self.f = np.zeros((Q,) + self.shape)          # f^eq at rest with p = 0
        self.g = self._scalar_eq3(phi0, z, z, z, p.eta_phi)
        self.h = self._scalar_eq3(psi0, z, z, z, p.eta_psi)
        self.first = True
        self.n = 0
        self.R_prev_phi = self.R_prev_psi = self.phiu_prev = self.psiu_prev = None
        self.H0 = self._H(phi0)
        self.log = []

    @staticmethod
    def _scalar_eq3(c, ux, uy, uz, eta):
        cu = _CXf * ux + _CYf * uy + _CZf * uz
        eq = _Wf * eta * c + _Wf * c * cu / CS2
        eq[0] += (1.0 - eta) * c
        return eq

    def _wall_ghosts3(self, phi, psi):
        """Ghost planes below y = 0 and above y = ny - 1 (Eq. boundary), from the wall planes."""
        return [self._ghost_values(w, phi[:, row, :], psi[:, row, :]) for w, row in ((0, 0), (1, self.ny - 1))]

    def _evaluate(self):
        p, d = self.p, self.d
        sh = self.shape
        phi = self.g.sum(axis=0)
        psi = self.h.sum(axis=0) if p.psi_on else np.zeros(sh)
        (phiGb, psiGb), (phiGt, psiGt) = self._wall_ghosts3(phi, psi)
        LG_phi = laplacian3(pad3(phi, phiGb, phiGt), sh)
        LN_phi = laplacian3(pad3(phi, phi[:, 0], phi[:, -1]), sh)
        LG_psi = laplacian3(pad3(psi, psiGb, psiGt), sh)
        LN_psi = laplacian3(pad3(psi, psi[:, 0], psi[:, -1]), sh)
        mu_phi = 4.0 * d.beta * (1.0 - psi) * (phi ** 3 - phi) - d.kappa * LG_phi + d.W * psi * phi
        if p.psi_on:
            psc = self._clamp(psi)
            clamps = int(np.count_nonzero(psc != psi))
            logterm = np.log(psc / (1.0 - psc))
            mu_psi = d.kT * logterm - d.lambda_s * LG_psi - d.beta * (1.0 - phi ** 2) ** 2 + 0.5 * d.W * phi ** 2
        else:
            clamps, logterm, mu_psi = 0, np.zeros(sh), np.zeros(sh)
        hp = np.ones(sh) if p.constraint == "linear" else self._gprime(phi)
        S1, S2 = float(np.sum(hp * mu_phi)), float(np.sum(hp * hp))
        Hval = self._H(phi)
        lam = 0.0
        if S2 > 0.0:
            lam = S1 / S2
            if p.multiplier == "target" and d.M_phi > 0.0:
                lam = (S1 + (self.H0 - Hval) / d.M_phi) / S2
        mubar = float(np.mean(mu_psi)) if p.psi_on else 0.0
        gm = gradient3(pad3(mu_phi, mu_phi[:, 0], mu_phi[:, -1]), sh)
        gp = gradient3(pad3(mu_psi, mu_psi[:, 0], mu_psi[:, -1]), sh)
        G = (p.Gx, p.Gy, 0.0)
        F = [-phi * gm[a] - psi * gp[a] + G[a] for a in range(3)]
        chi = np.clip(0.5 * (phi / d.phi_b + 1.0), 0.0, 1.0)
        rho = p.rho_g + (p.rho_l - p.rho_g) * chi
        gr = gradient3(pad3(rho, rho[:, 0], rho[:, -1]), sh)
        f = self.f
        j = [np.tensordot(c.astype(np.float64), f, axes=(0, 0)) for c in (CX, CY, CZ)]
        u = [(j[a] + 0.5 * F[a]) / rho for a in range(3)]
        usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
        ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2]
        pres = CS2 / (1.0 - W[0]) * (f[1:].sum(axis=0) + 0.5 * ugr - rho * W[0] * usq / (2.0 * CS2))
        return dict(phi=phi, psi=psi, LG_phi=LG_phi, LN_phi=LN_phi, LG_psi=LG_psi, LN_psi=LN_psi,
                    mu_phi=mu_phi, mu_psi=mu_psi, logterm=logterm, hp=hp, S1=S1, S2=S2, H=Hval, lam=lam,
                    mubar=mubar, F=F, rho=rho, gr=gr, chi=chi, u=u, usq=usq, ugr=ugr, p=pres, clamps=clamps,
                    ghosts=((phiGb, psiGb), (phiGt, psiGt)))

    def _stream_flow3(self, post, rho):
        ny = self.ny
        new = np.empty_like(post)
        for k in range(Q):
            sh = np.roll(np.roll(post[k], CX[k], axis=2), CZ[k], axis=0)
            if CY[k] == 0:
                new[k] = sh
                continue
            o = OPP[k]
            if CY[k] == 1:
                new[k][:, 1:] = sh[:, :-1]
                row, wall = 0, self.p.walls[0]
            else:
                new[k][:, :-1] = sh[:, 1:]
                row, wall = ny - 1, self.p.walls[1]
            new[k][:, row] = post[o][:, row] - 2.0 * W[o] * rho[:, row] * CX[o] * wall.u_x / CS2
        return new

    def _stream_scalar3(self, post):
        ny = self.ny
        new = np.empty_like(post)
        for k in range(Q):
            sh = np.roll(np.roll(post[k], CX[k], axis=2), CZ[k], axis=0)
            if CY[k] == 0:
                new[k] = sh
                continue
            shm = np.roll(np.roll(post[MIRY[k]], CX[k], axis=2), CZ[k], axis=0)
            if CY[k] == 1:
                new[k][:, 1:] = sh[:, :-1]
                new[k][:, 0] = shm[:, 0]
            else:
                new[k][:, :-1] = sh[:, 1:]
                new[k][:, ny - 1] = shm[:, ny - 1]
        return new

    def _one(self):
        p, d = self.p, self.d
        e = self._evaluate()
        phi, psi, rho = e["phi"], e["psi"], e["rho"]
        ux, uy, uz = e["u"]
        cu = _CXf * ux + _CYf * uy + _CZf * uz
        feq = (e["p"] / CS2) * _Wf + rho * _Wf * (cu / CS2 + cu * cu / (2 * CS2 ** 2) - e["usq"] / (2 * CS2))
        feq[0] -= e["p"] / CS2
        geq = self._scalar_eq3(phi, ux, uy, uz, p.eta_phi)
        heq = self._scalar_eq3(psi, ux, uy, uz, p.eta_psi)
        Fx, Fy, Fz = e["F"]
        cF = _CXf * Fx + _CYf * Fy + _CZf * Fz
        cgr = _CXf * e["gr"][0] + _CYf * e["gr"][1] + _CZf * e["gr"][2]
        src_f = _Wf * (e["ugr"] + cF / CS2 + (cu * cgr - CS2 * e["ugr"]) / CS2)
        R_phi = d.M_phi * (-4.0 * d.beta * (1.0 - psi) * (phi ** 3 - phi) - d.W * psi * phi + e["lam"] * e["hp"]) \
            + d.M_phi * d.kappa * (e["LG_phi"] - e["LN_phi"])
        if p.psi_on:
            R_psi = (d.M_psi * (-d.kT * e["logterm"] + d.beta * (1.0 - phi ** 2) ** 2 - 0.5 * d.W * phi ** 2
                                + e["mubar"])
                     + d.M_psi * d.lambda_s * (e["LG_psi"] - e["LN_psi"]) - d.M_0 * e["LN_psi"])
        else:
            R_psi = np.zeros(self.shape)
        phiu = np.stack([phi * ux, phi * uy, phi * uz])
        psiu = np.stack([psi * ux, psi * uy, psi * uz])
        if self.first:
            self.R_prev_phi, self.R_prev_psi = R_phi, R_psi
            self.phiu_prev, self.psiu_prev = phiu, psiu
        dphiu, dpsiu = phiu - self.phiu_prev, psiu - self.psiu_prev
        srcA_g = _Wf * (_CXf * dphiu[0] + _CYf * dphiu[1] + _CZf * dphiu[2]) / CS2
        srcA_h = _Wf * (_CXf * dpsiu[0] + _CYf * dpsiu[1] + _CZf * dpsiu[2]) / CS2
        nu = d.nu_g + (d.nu_l - d.nu_g) * e["chi"]
        s_f = 1.0 / (nu / CS2 + 0.5)
        s_g, s_h = 1.0 / p.tau_g, 1.0 / p.tau_h
        fpost = self.f - s_f * (self.f - feq) + (1.0 - 0.5 * s_f) * src_f
        gpost = self.g - s_g * (self.g - geq) + (1.0 - 0.5 * s_g) * srcA_g + _Wf * (1.5 * R_phi - 0.5 * self.R_prev_phi)
        if p.psi_on:
            hpost = (self.h - s_h * (self.h - heq) + (1.0 - 0.5 * s_h) * srcA_h
                     + _Wf * (1.5 * R_psi - 0.5 * self.R_prev_psi))
        else:
            hpost = np.zeros_like(self.h)
        self.f = self._stream_flow3(fpost, rho)
        self.g = self._stream_scalar3(gpost)
        self.h = self._stream_scalar3(hpost)
        self.R_prev_phi, self.R_prev_psi = R_phi, R_psi
        self.phiu_prev, self.psiu_prev = phiu, psiu
        self.first = False
        self.log.append(dict(n=self.n, lam=e["lam"], mubar=e["mubar"], H=e["H"], psi_total=float(np.sum(psi)),
                             phi_total=float(np.sum(phi)), kinetic=float(np.sum(0.5 * rho * e["usq"]))))
        self.n += 1

    def fields(self):
        """phi, psi, u_x, u_y, u_z, p at the current time, [z][y][x]."""
        e = self._evaluate()
        ux, uy, uz = e["u"]
        return {"phi": e["phi"].copy(), "psi": e["psi"].copy(), "ux": ux.copy(), "uy": uy.copy(),
                "uz": uz.copy(), "p": e["p"].copy()}

    def totals(self):
        e = self._evaluate()
        phi, psi = e["phi"], e["psi"]
        return dict(step=self.n, Q=float(np.sum(2.0 * self._g(phi))), H=e["H"], psi_total=float(np.sum(psi)),
                    phi_total=float(np.sum(phi)), lam=e["lam"], mubar=e["mubar"],
                    kinetic=float(np.sum(0.5 * e["rho"] * e["usq"])), clamps=e["clamps"])
