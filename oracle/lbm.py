"""The coupled MRT lattice Boltzmann step, written out in numpy float64 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

One call of ``Oracle.step`` advances every field by one time step in the order of
the textbook collide-then-stream form of the paper's unified evolution equation
(Sec. 3):

    f_{i,k}(x + c_i dt, t + dt) = f_{i,k} - (M^-1 S^k M)_{ij} (f_{j,k} - f^eq_{j,k}) + dt F_{i,k}

with k = flow (f), phase field (g) and surfactant (h).  The state held between
steps is the set of pre-collision populations at time t plus the backward-difference
history needed by the source terms.  Each step:

1.  moments phi = sum g, psi = sum h (Sec. 3, macroscopic quantities);
2.  wall ghost rows for phi, psi from the natural boundary conditions (Eq. boundary,
    closed by ghost rows as below);
3.  chemical potentials mu_phi, mu_psi (Eqs. eq_muphi, eq_mupsi) with the isotropic
    Laplacian (Sec. 3, stencils);
4.  the Lagrange multipliers lambda_phi = int h' mu / int h'^2 (Eq. eq15) and
    mubar_psi = mean(mu_psi) (Eq. AC_psi);
5.  the force F = -phi grad mu_phi - psi grad mu_psi + G (Eq. eq_Fs0), velocity and
    pressure (Sec. 3, macroscopic quantities);
6.  equilibria, source terms and the MRT collision of all three sets (Sec. 3);
7.  streaming: halfway bounce-back with the moving-wall term for the flow set,
    specular reflection for the two scalar sets.

Wall closure (the paper cites an external scheme and does not print it):
ghost rows phi_G = phi_0 - (df_w/dphi)/kappa and psi_G = psi_0 - (df_w/dpsi)/lambda_s
evaluated with the wall-row values; mu and rho use mirror ghosts.  Because
bounce-back gives the lattice diffusion a zero wall flux, the wall flux of the
natural boundary condition enters R as kappa-weighted (Lap_G - Lap_N) terms, which
are zero away from the walls.
"""

import math
import numpy as np

from .lattice import CX, CY, W, OPP, MIRY, CS2, Q, moment_matrix, rate_vector
from .params import derive

_CXf = CX.astype(np.float64)[:, None, None]
_CYf = CY.astype(np.float64)[:, None, None]
_Wf = W[:, None, None]


def _neighbor(P, k, ny, nx):
    """Value at x + c_k taken from an (ny+2, nx+2) array padded by one ghost ring."""
    return P[1 + CY[k]:1 + CY[k] + ny, 1 + CX[k]:1 + CX[k] + nx]


def _pad(a, bottom, top):
    """Pad with ghost rows below row 0 and above row ny-1; x wraps periodically."""
    ny, nx = a.shape
    P = np.empty((ny + 2, nx + 2))
    P[1:-1, 1:-1] = a
    P[0, 1:-1] = bottom
    P[-1, 1:-1] = top
    P[:, 0] = P[:, -2]
    P[:, -1] = P[:, 1]
    return P


def laplacian(P, ny, nx):
    """Isotropic Laplacian: sum_{i!=0} 2 w_i [z(x+c_i) - z(x)] / c_s^2 (Sec. 3)."""
    c = P[1:-1, 1:-1]
    out = np.zeros((ny, nx))
    for k in range(1, Q):
        out += W[k] * (_neighbor(P, k, ny, nx) - c)
    return 2.0 * out / CS2


def gradient(P, ny, nx):
    """Isotropic gradient: sum_{i!=0} w_i c_i z(x+c_i) / c_s^2 (Sec. 3)."""
    gx = np.zeros((ny, nx))
    gy = np.zeros((ny, nx))
    for k in range(1, Q):
        nb = _neighbor(P, k, ny, nx)
        gx += W[k] * CX[k] * nb
        gy += W[k] * CY[k] * nb
    return gx / CS2, gy / CS2


class Oracle:
    """Plain FP64 implementation of the paper's coupled LBM (Sec. 3) on a channel:
    x periodic, halfway bounce-back walls below row 0 and above row ny-1."""

    def __init__(self, params, phi0, psi0=None, u0=(0.0, 0.0), source=None, force=True):
        """u0: uniform initial velocity (the equilibria of the initial state carry it);
        source: optional callable n -> (S_phi, S_psi), arrays added to R_phi, R_psi of step
        n (a manufactured source, lattice units per step); force=False: no force acts on
        the flow (with walls sliding at u0 the flow stays uniform, a prescribed velocity)."""
        p = params
        self.p = p
        self.source = source
        self.force = force
        self.d = derive(p)
        self.ny, self.nx = p.ny, p.nx
        if p.ny < 2 or p.nx < 1:
            raise ValueError("grid must have nx >= 1 and ny >= 2")
        phi0 = np.asarray(phi0, dtype=np.float64)
        if phi0.shape != (p.ny, p.nx):
            raise ValueError("phi0 must be (ny, nx)")
        if psi0 is None or not p.psi_on:
            psi0 = np.zeros_like(phi0)
        psi0 = np.asarray(psi0, dtype=np.float64)
        self.Mm = moment_matrix()
        self.Minv = np.linalg.inv(self.Mm)
        # pre-collision populations at t = 0: equilibria of the initial fields with p = 0
        # and the uniform velocity u0 (f^eq vanishes identically at rest)
        ux0 = np.full_like(phi0, float(u0[0]))
        uy0 = np.full_like(phi0, float(u0[1]))
        rho0 = p.rho_g + (p.rho_l - p.rho_g) * np.clip(0.5 * (phi0 / self.d.phi_b + 1.0), 0.0, 1.0)
        cu0 = _CXf * ux0 + _CYf * uy0
        self.f = rho0 * _Wf * (cu0 / CS2 + cu0 * cu0 / (2 * CS2 ** 2) - (ux0 * ux0 + uy0 * uy0) / (2 * CS2))
        self.g = self._scalar_eq(phi0, ux0, uy0, p.eta_phi)
        self.h = self._scalar_eq(psi0, ux0, uy0, p.eta_psi)
        self.first = True
        self.n = 0
        self.R_prev_phi = None
        self.R_prev_psi = None
        self.phiu_prev = None
        self.psiu_prev = None
        self.H0 = self._H(phi0)
        self.log = []

    # ------------------------------------------------------------------ helpers
    @staticmethod
    def _scalar_eq(c, ux, uy, eta):
        """f^eq_{i,2} / f^eq_{i,3} of Sec. 3."""
        cu = _CXf * ux + _CYf * uy
        eq = _Wf * eta * c + _Wf * c * cu / CS2
        eq[0] += (1.0 - eta) * c
        return eq

    def _g(self, phi):
        pb = self.d.phi_b
        return 3.0 * phi / (4.0 * pb) - phi * phi * phi / (4.0 * pb * pb * pb)

    def _gprime(self, phi):
        pb = self.d.phi_b
        return 3.0 / (4.0 * pb) - 3.0 * phi ** 2 / (4.0 * pb * pb * pb)

    def _H(self, phi):
        """The conserved functional sum h_phi(phi): h = 1/2 + g (nonlinear) or phi (linear)."""
        if self.p.constraint == "linear":
            return float(np.sum(phi))
        return float(np.sum(0.5 + self._g(phi)))

    def _clamp(self, psi):
        e = self.p.psi_clamp
        return np.clip(psi, e, 1.0 - e)

    def _wall_tension_factors(self, w, L):
        """t_a = sigma_s,a / sigma_s,a,0 - 1 of wall w for a in (sg, sl), and whether the
        logarithmic law is in force: t_a = beta_a L (Eq. langmuir, L = ln(1 - psi)), capped
        at -1/2 where the tension would fall below half its clean value (Remark 1) when
        p.saturation; on_a = 1 where dt_a/dpsi = -beta_a / (1 - psi), 0 on the cap."""
        wl = self.p.walls[w]
        t_sg, t_sl = wl.beta_sg * L, wl.beta_sl * L
        if not self.p.saturation:
            return t_sg, t_sl, 1.0, 1.0
        on_sg, on_sl = t_sg > -0.5, t_sl > -0.5
        return np.where(on_sg, t_sg, -0.5), np.where(on_sl, t_sl, -0.5), on_sg, on_sl

    def _wall_ghosts(self, phi, psi):
        """Ghost rows (bottom at j = -1, top at j = ny) from Eq. boundary."""
        return [self._ghost_values(w, phi[row], psi[row]) for w, row in ((0, 0), (1, self.ny - 1))]

    def _ghost_values(self, w, ph, ps):
        """Ghost values beyond wall w from the wall-row values ph, ps (any shape):
        phi_G = phi_0 - (df_w/dphi)/kappa, psi_G = psi_0 - (df_w/dpsi)/lambda_s."""
        d, p = self.d, self.p
        psc = self._clamp(ps) if p.psi_on else ps
        L = np.log1p(-psc)
        t_sg, t_sl, on_sg, on_sl = self._wall_tension_factors(w, L)
        # f_w = (1/2 - g) sigma_sg + (1/2 + g) sigma_sl with sigma_s,a = sigma_s,a,0 (1 + t_a)
        # and sigma_sg,0 - sigma_sl,0 written as sigma cos(theta0) (Eq. fw0, Eq. langmuir)
        dfdphi = -(d.wall_cos[w] + d.wall_sg0[w] * t_sg - d.wall_sl0[w] * t_sl) * self._gprime(ph)
        g = self._g(ph)
        dfdpsi = -((0.5 - g) * d.wall_sg0[w] * p.walls[w].beta_sg * on_sg
                   + (0.5 + g) * d.wall_sl0[w] * p.walls[w].beta_sl * on_sl) / (1.0 - psc)
        phiG = ph - dfdphi / d.kappa if d.kappa > 0 else ph.copy()
        psiG = ps - dfdpsi / d.lambda_s if (d.lambda_s > 0 and p.psi_on) else ps.copy()
        return phiG, psiG

    def _rates(self, main, others, shape, flow):
        """Per-cell diagonal of S (9, ny, nx); zeros in ``others`` mean 'equal to main'."""
        main = np.broadcast_to(np.asarray(main, dtype=np.float64), shape)
        o = [main if v == 0 else np.full(shape, float(v)) for v in others]
        if flow:   # others = (s0, s1, s3, s4), main = s2 (viscous)
            s = [o[0], o[1], o[1], main, main, main, o[2], o[2], o[3]]
        else:      # others = (s0, s2, s3, s4), main = s1 (diffusive)
            s = [o[0], main, main, o[1], o[1], o[1], o[2], o[2], o[3]]
        return np.stack(s)

    def _lambda_weight(self):
        """Weight of R^n in the source 1.5 R^n - 0.5 R^{n-1}; 1 on the first step, where
        the history starts from R^{-1} := R^0."""
        return 1.0 if self.first else 1.5

    def _exact_lambda(self, A, B, lam_est):
        """The root of H(A + lambda B) = H(phi^0) nearest the continuous estimate: a cubic
        in lambda for the nonlinear constraint (h = 1/2 + g, g cubic in phi), linear for
        the linear one.  Coefficients are the exact expansion of g(A + lambda B)."""
        pb = self.d.phi_b
        if self.p.constraint == "linear":
            coef = [float(np.sum(B)), float(np.sum(A)) - self.H0]
        else:
            k1, k3 = 3.0 / (4.0 * pb), 1.0 / (4.0 * pb ** 3)
            coef = [float(np.sum(-k3 * B ** 3)),
                    float(np.sum(-3.0 * k3 * A * B * B)),
                    float(np.sum(k1 * B - 3.0 * k3 * A * A * B)),
                    float(np.sum(0.5 + k1 * A - k3 * A ** 3)) - self.H0]
        roots = np.roots(coef)
        real = roots[np.abs(roots.imag) <= 1e-9 * np.maximum(1.0, np.abs(roots.real))].real
        if real.size == 0:
            raise FloatingPointError("no real multiplier conserves H")
        return float(real[np.argmin(np.abs(real - lam_est))])

    def _collide(self, pop, eq, s, src):
        """pop - M^-1 S M (pop - eq) + M^-1 (I - S/2) M src   (Sec. 3, A^k)."""
        m = np.tensordot(self.Mm, pop - eq, axes=(1, 0)) * s
        ms = np.tensordot(self.Mm, src, axes=(1, 0)) * (1.0 - 0.5 * s)
        return pop - np.tensordot(self.Minv, m, axes=(1, 0)) + np.tensordot(self.Minv, ms, axes=(1, 0))

    def _stream_flow(self, post, rho):
        """Pull streaming of the flow set: f_k(x) = f*_k(x - c_k); a link whose source
        lies in a wall bounces back, f_k(x) = f*_o(x) - 2 w_o rho (c_o . u_w) / c_s^2
        with o the opposite direction (halfway bounce-back, moving wall)."""
        ny = self.ny
        new = np.empty_like(post)
        for k in range(Q):
            sh = np.roll(post[k], CX[k], axis=1)
            if CY[k] == 0:
                new[k] = sh
                continue
            o = OPP[k]
            if CY[k] == 1:
                new[k, 1:] = sh[:-1]
                row, wall = 0, self.p.walls[0]
            else:
                new[k, :-1] = sh[1:]
                row, wall = ny - 1, self.p.walls[1]
            new[k, row] = post[o, row] - 2.0 * W[o] * rho[row] * CX[o] * wall.u_x / CS2
        return new

    def _stream_scalar(self, post):
        """Pull streaming of a scalar set with specular walls: a link whose
        source lies in a wall takes the population that left the mirror node toward the
        wall, i.e. g_k(x) = g*_m(x - (c_kx, 0)) with m the direction (c_kx, -c_ky).
        This is a zero normal flux that keeps the tangential flux of the diagonal links,
        so the lattice diffusion at a wall row is the mirror-ghost Laplacian."""
        ny = self.ny
        new = np.empty_like(post)
        for k in range(Q):
            sh = np.roll(post[k], CX[k], axis=1)
            if CY[k] == 0:
                new[k] = sh
                continue
            m = MIRY[k]
            shm = np.roll(post[m], CX[k], axis=1)
            if CY[k] == 1:
                new[k, 1:] = sh[:-1]
                new[k, 0] = shm[0]
            else:
                new[k, :-1] = sh[1:]
                new[k, ny - 1] = shm[ny - 1]
        return new

    # --------------------------------------------------------------- evaluation
    def _evaluate(self):
        """Steps 1-5 at the current pre-collision state; pure (no state change)."""
        p, d = self.p, self.d
        ny, nx = self.ny, self.nx
        e = {}
        phi = self.g.sum(axis=0)
        psi = self.h.sum(axis=0) if p.psi_on else np.zeros((ny, nx))
        (phiGb, psiGb), (phiGt, psiGt) = self._wall_ghosts(phi, psi)
        phiP_G = _pad(phi, phiGb, phiGt)
        psiP_G = _pad(psi, psiGb, psiGt)
        phiP_N = _pad(phi, phi[0], phi[-1])
        psiP_N = _pad(psi, psi[0], psi[-1])
        LG_phi = laplacian(phiP_G, ny, nx)
        LN_phi = laplacian(phiP_N, ny, nx)
        LG_psi = laplacian(psiP_G, ny, nx)
        LN_psi = laplacian(psiP_N, ny, nx)

        # chemical potentials (Eqs. eq_muphi, eq_mupsi)
        mu_phi = 4.0 * d.beta * (1.0 - psi) * (phi * phi * phi - phi) - d.kappa * LG_phi + d.W * psi * phi
        if p.psi_on:
            psc = self._clamp(psi)
            clamps = int(np.count_nonzero(psc != psi))
            logterm = np.log(psc / (1.0 - psc))
            mu_psi = (d.kT * logterm - d.lambda_s * LG_psi - d.beta * (1.0 - phi ** 2) ** 2
                      + 0.5 * d.W * phi ** 2)
        else:
            clamps = 0
            logterm = np.zeros((ny, nx))
            mu_psi = np.zeros((ny, nx))

        # Lagrange multipliers (Eqs. eq15, AC_psi, AC_phi)
        if p.constraint == "linear":
            hp = np.ones((ny, nx))
        else:
            hp = self._gprime(phi)
        S1 = float(np.sum(hp * mu_phi))
        S2 = float(np.sum(hp * hp))
        Hval = self._H(phi)
        if S2 > 0.0:
            lam = S1 / S2
            if p.multiplier == "target" and d.M_phi > 0.0:
                lam = (S1 + (self.H0 - Hval) / d.M_phi) / S2
        else:
            lam = 0.0
        mubar = float(np.mean(mu_psi)) if p.psi_on else 0.0

        # force (Eq. eq_Fs0), density, velocity and pressure (Sec. 3)
        muP = _pad(mu_phi, mu_phi[0], mu_phi[-1])
        mpP = _pad(mu_psi, mu_psi[0], mu_psi[-1])
        gmx, gmy = gradient(muP, ny, nx)
        gpx, gpy = gradient(mpP, ny, nx)
        if self.force:
            Fx = -phi * gmx - psi * gpx + p.Gx
            Fy = -phi * gmy - psi * gpy + p.Gy
        else:
            Fx = np.zeros((ny, nx))
            Fy = np.zeros((ny, nx))
        # liquid fraction, clipped to [0, 1]: the bulk |phi| exceeds phi_b(psi_b) wherever
        # the bulk surfactant falls below psi_b (Sec. 2.2), and rho, nu stay within the
        # pure-phase values (at rho_l / rho_g = 1000 an unclipped chi of -1e-3 gives rho ~ 0)
        chi = np.clip(0.5 * (phi / d.phi_b + 1.0), 0.0, 1.0)
        rho = p.rho_g + (p.rho_l - p.rho_g) * chi
        grx, gry = gradient(_pad(rho, rho[0], rho[-1]), ny, nx)
        f = self.f
        jx = np.tensordot(CX.astype(np.float64), f, axes=(0, 0))
        jy = np.tensordot(CY.astype(np.float64), f, axes=(0, 0))
        ux = (jx + 0.5 * Fx) / rho
        uy = (jy + 0.5 * Fy) / rho
        usq = ux * ux + uy * uy
        ugr = ux * grx + uy * gry
        pres = CS2 / (1.0 - W[0]) * (f[1:].sum(axis=0) + 0.5 * ugr - rho * W[0] * usq / (2.0 * CS2))

        e.update(phi=phi, psi=psi, LG_phi=LG_phi, LN_phi=LN_phi, LG_psi=LG_psi, LN_psi=LN_psi,
                 mu_phi=mu_phi, mu_psi=mu_psi, logterm=logterm, hp=hp, S1=S1, S2=S2, H=Hval,
                 lam=lam, mubar=mubar, Fx=Fx, Fy=Fy, rho=rho, grx=grx, gry=gry, chi=chi,
                 ux=ux, uy=uy, usq=usq, ugr=ugr, p=pres, clamps=clamps,
                 ghosts=((phiGb, psiGb), (phiGt, psiGt)))
        return e

    # --------------------------------------------------------------------- step
    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            self._one()

    def _one(self):
        p, d = self.p, self.d
        ny, nx = self.ny, self.nx
        e = self._evaluate()
        phi, psi, ux, uy, rho = e["phi"], e["psi"], e["ux"], e["uy"], e["rho"]

        # equilibria (Sec. 3)
        cu = _CXf * ux + _CYf * uy
        feq = (e["p"] / CS2) * _Wf + rho * _Wf * (cu / CS2 + cu * cu / (2 * CS2 ** 2) - e["usq"] / (2 * CS2))
        feq[0] -= e["p"] / CS2
        geq = self._scalar_eq(phi, ux, uy, p.eta_phi)
        heq = self._scalar_eq(psi, ux, uy, p.eta_psi)

        # flow source, literal form of F_{i,1} (Sec. 3)
        cF = _CXf * e["Fx"] + _CYf * e["Fy"]
        cgr = _CXf * e["grx"] + _CYf * e["gry"]
        bracket = e["ugr"] + cF / CS2 + (cu * cgr - CS2 * e["ugr"]) / CS2
        src_f = _Wf * bracket

        # reaction terms R_phi, R_psi (Sec. 3) with the kappa-weighted wall flux of the ghost-row closure
        R_phi = d.M_phi * (-4.0 * d.beta * (1.0 - psi) * (phi * phi * phi - phi) - d.W * psi * phi
                           + e["lam"] * e["hp"]) + d.M_phi * d.kappa * (e["LG_phi"] - e["LN_phi"])
        if p.psi_on:
            R_psi = (d.M_psi * (-d.kT * e["logterm"] + d.beta * (1.0 - phi ** 2) ** 2
                                - 0.5 * d.W * phi ** 2 + e["mubar"])
                     + d.M_psi * d.lambda_s * (e["LG_psi"] - e["LN_psi"]) - d.M_0 * e["LN_psi"])
        else:
            R_psi = np.zeros((ny, nx))
        if self.source is not None:
            S_phi, S_psi = self.source(self.n)
            R_phi = R_phi + S_phi
            if p.psi_on:
                R_psi = R_psi + S_psi
        phiu = np.stack([phi * ux, phi * uy])
        psiu = np.stack([psi * ux, psi * uy])
        if self.first:   # first step: the backward differences start from zero
            self.R_prev_phi, self.R_prev_psi = R_phi, R_psi
            self.phiu_prev, self.psiu_prev = phiu, psiu
        dphiu = phiu - self.phiu_prev
        dpsiu = psiu - self.psiu_prev
        srcA_g = _Wf * (_CXf * dphiu[0] + _CYf * dphiu[1]) / CS2
        srcA_h = _Wf * (_CXf * dpsiu[0] + _CYf * dpsiu[1]) / CS2

        # relaxation rates: nu(phi) interpolated, tau = nu / c_s^2 + 1/2 (Sec. 3)
        nu = d.nu_g + (d.nu_l - d.nu_g) * e["chi"]
        s_f = self._rates(1.0 / (nu / CS2 + 0.5), p.mrt_f, (ny, nx), flow=True)
        s_g = self._rates(1.0 / p.tau_g, p.mrt_g, (ny, nx), flow=False)
        s_h = self._rates(1.0 / p.tau_h, p.mrt_h, (ny, nx), flow=False)

        fpost = self._collide(self.f, feq, s_f, src_f)
        if p.multiplier == "exact":
            # phi^{n+1} is affine in lambda^n: the multiplier enters the phi populations
            # only through w_i a M_phi lambda h' (a = 1.5, or 1 on the first step, where
            # R^{n-1} := R^n); stream the two parts separately and choose lambda so that
            # the discrete H(phi^{n+1}) equals H(phi^0) (Sec. 2, the constraint in its
            # discrete form)
            a = self._lambda_weight()
            lam_part = d.M_phi * e["lam"] * e["hp"]
            R0 = R_phi - lam_part
            Rp = R0 if self.first else self.R_prev_phi
            gA = self._stream_scalar(self._collide(self.g, geq, s_g, srcA_g) + _Wf * (1.5 * R0 - 0.5 * Rp))
            gB = self._stream_scalar(_Wf * (a * d.M_phi * e["hp"]))
            lam = self._exact_lambda(gA.sum(axis=0), gB.sum(axis=0), e["lam"])
            e["lam_paper"] = e["lam"]
            e["lam"] = lam
            R_phi = R0 + d.M_phi * lam * e["hp"]
            if self.first:
                self.R_prev_phi = R_phi
            gnew = gA + lam * gB
        gpost = self._collide(self.g, geq, s_g, srcA_g) + _Wf * (1.5 * R_phi - 0.5 * self.R_prev_phi)
        if p.psi_on:
            hpost = self._collide(self.h, heq, s_h, srcA_h) + _Wf * (1.5 * R_psi - 0.5 * self.R_prev_psi)
        else:
            hpost = np.zeros_like(self.h)

        self.f = self._stream_flow(fpost, rho)
        self.g = gnew if p.multiplier == "exact" else self._stream_scalar(gpost)
        self.h = self._stream_scalar(hpost)
        self.R_prev_phi, self.R_prev_psi = R_phi, R_psi
        self.phiu_prev, self.psiu_prev = phiu, psiu
        self.first = False
        self.log.append(dict(n=self.n, lam=e["lam"], lam_paper=e.get("lam_paper", e["lam"]),
                             mubar=e["mubar"], S1=e["S1"], S2=e["S2"],
                             H=e["H"], Q=float(np.sum(2.0 * self._g(phi))), psi_total=float(np.sum(psi)),
                             phi_total=float(np.sum(phi)), kinetic=float(np.sum(0.5 * rho * e["usq"])),
                             clamps=e["clamps"]))
        self.n += 1

    # -------------------------------------------------------------- diagnostics
    def fields(self):
        """phi, psi, u_x, u_y, p at the current time (moments of the current state)."""
        e = self._evaluate()
        return {k: e[k].copy() for k in ("phi", "psi", "ux", "uy", "p")}

    def totals(self):
        """Conserved and reduced quantities at the current time."""
        e = self._evaluate()
        phi, psi = e["phi"], e["psi"]
        return dict(step=self.n, Q=float(np.sum(2.0 * self._g(phi))), H=e["H"],
                    psi_total=float(np.sum(psi)), phi_total=float(np.sum(phi)),
                    lam=e["lam"], mubar=e["mubar"], kinetic=float(np.sum(0.5 * e["rho"] * e["usq"])),
                    free_energy=self.free_energy(e), clamps=e["clamps"])

    def free_energy(self, e=None):
        """Discrete E_f of Eq. eq1: cell sums of the bulk densities and of
        kappa/2 |grad phi|^2, lambda_s/2 |grad psi|^2 (isotropic gradient with the
        wetting ghosts) plus the wall energy f_w of Eq. eq8 on both walls."""
        if e is None:
            e = self._evaluate()
        d, p = self.d, self.p
        ny, nx = self.ny, self.nx
        phi, psi = e["phi"], e["psi"]
        (phiGb, psiGb), (phiGt, psiGt) = e["ghosts"]
        gx, gy = gradient(_pad(phi, phiGb, phiGt), ny, nx)
        bulk = d.beta * (phi ** 2 - 1.0) ** 2 + 0.5 * d.kappa * (gx * gx + gy * gy)
        if p.psi_on:
            psc = self._clamp(psi)
            sx, sy = gradient(_pad(psi, psiGb, psiGt), ny, nx)
            bulk = bulk + d.kT * (psc * np.log(psc) + (1.0 - psc) * np.log1p(-psc)) \
                + 0.5 * d.lambda_s * (sx * sx + sy * sy) \
                - d.beta * psi * (1.0 - phi ** 2) ** 2 + 0.5 * d.W * psi * phi ** 2
        E = float(np.sum(bulk))
        for w, row in ((0, 0), (1, ny - 1)):
            ph = phi[row]
            ps = self._clamp(psi[row]) if p.psi_on else psi[row]
            L = np.log1p(-ps)
            s_sum = 16.0 * p.sigma / 15.0
            t_sg, t_sl, _, _ = self._wall_tension_factors(w, L)
            fw = (-(d.wall_cos[w] + d.wall_sg0[w] * t_sg - d.wall_sl0[w] * t_sl) * self._g(ph)
                  + 0.5 * (d.wall_sg0[w] * t_sg + d.wall_sl0[w] * t_sl) + 0.5 * s_sum)
            E += float(np.sum(fw))
        return E
