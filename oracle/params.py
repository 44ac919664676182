"""Parameters of the coupled model and their lattice-unit derivation (oracle side).

All quantities are lattice units (dx = dt = 1, c_s^2 = 1/3).  Grid nodes (i, j)
sit at x = i, y = j + 1/2; x is periodic and the two walls lie half a spacing
below row 0 (y = 0) and above row ny-1 (y = ny).

Derivations, each from the paper:
* kappa = 3 eps sigma / 8 and beta = 3 sigma / (4 eps)                (Sec. 2.1, E_GL)
* lambda_s = kappa / 2                                                 (Sec. 2.1, E_sur)
* Ex = 4 beta / W and Pi = k_B T / (4 beta)                            (Sec. 4, dimensionless groups)
* phi_b^2 = 1 - W psi_b / (4 beta (1 - psi_b))                          (Sec. 2.2)
* g(phi) = 3 phi / (4 phi_b) - phi^3 / (4 phi_b^3), h_phi = 1/2 + g      (Sec. 2.1, Eq. AC_phi)
* sigma_sg0 - sigma_sl0 = sigma cos(theta0), sigma_sg0 + sigma_sl0 = 16 sigma / 15
                                                                       (Sec. 4.4 worked values)
* nu = c_s^2 (1/s2^1 - 1/2); M_phi kappa = eta_phi c_s^2 (1/s1^2 - 1/2);
  M_psi lambda_s + M_0 = eta_psi c_s^2 (1/s1^3 - 1/2)                   (Sec. 3, relaxation rates)

Readings where the paper is silent: M_0 is whatever the
last relation leaves once M_psi is chosen; rho and nu interpolate linearly in
(phi/phi_b + 1)/2; eta_phi = eta_psi = 1 by default; unspecified MRT rates equal
the field's main rate.
"""

from dataclasses import dataclass, field
import math

CS2 = 1.0 / 3.0


@dataclass
class Wall:
    """One solid wall: clean contact angle (degrees), solid adsorption elasticities
    beta_sg, beta_sl (Eq. langmuir) and tangential wall speed u_x."""

    theta0_deg: float = 90.0
    beta_sg: float = 0.0
    beta_sl: float = 0.0
    u_x: float = 0.0


@dataclass
class OracleParams:
    nx: int
    ny: int
    tau_f: float = 0.8           # flow relaxation time of the liquid, 1/s2^1
    tau_f_gas: float = -1.0      # <= 0: same as tau_f
    tau_g: float = 0.8           # phase field, 1/s1^2
    tau_h: float = 0.8           # surfactant, 1/s1^3
    # remaining MRT rates, ordered (s0, s1, s3, s4) for flow and (s0, s2, s3, s4) for
    # the scalars; 0 means "equal to the field's main rate" (BGK when all are 0)
    mrt_f: tuple = (0.0, 0.0, 0.0, 0.0)
    mrt_g: tuple = (0.0, 0.0, 0.0, 0.0)
    mrt_h: tuple = (0.0, 0.0, 0.0, 0.0)
    sigma: float = 0.01          # clean gas-liquid tension sigma_gl,0
    eps: float = 4.0             # interface thickness parameter epsilon
    Ex: float = 1.0              # solubility parameter (<= 0 means W = 0)
    Pi: float = 0.18407          # thermal parameter k_B T / (4 beta)
    M_phi: float = 0.0           # used only when kappa == 0 (otherwise derived)
    M_psi: float = 0.5
    eta_phi: float = 1.0
    eta_psi: float = 1.0
    lambda_s: float = -1.0       # < 0: kappa / 2
    psi_b: float = 0.0           # reference bulk surfactant for phi_b
    phi_b: float = -1.0          # <= 0: derived from psi_b
    rho_l: float = 1.0
    rho_g: float = 1.0
    Gx: float = 0.0              # body-force density
    Gy: float = 0.0
    constraint: str = "nonlinear"   # "nonlinear" (h_phi = 1/2 + g) or "linear" (h_phi = phi)
    multiplier: str = "paper"       # "paper" (Eq. eq15), "target" (drift-correcting reading) or
                                    # "exact" (the root of the discrete constraint H(phi^{n+1}) = H(phi^0))
    psi_on: bool = True             # False: surfactant transport disabled, psi == 0
    walls: list = field(default_factory=lambda: [Wall(), Wall()])  # [bottom, top]
    psi_clamp: float = 1e-12
    saturation: bool = True         # Remark 1 cap: sigma_s,alpha >= sigma_s,alpha,0 / 2


@dataclass
class Derived:
    beta: float
    kappa: float
    lambda_s: float
    W: float
    kT: float
    phi_b: float
    M_phi: float
    M_psi: float
    M_0: float
    nu_l: float
    nu_g: float
    wall_A: list   # sigma_sg0 beta_sg - sigma_sl0 beta_sl per wall
    wall_B: list   # sigma_sg0 beta_sg + sigma_sl0 beta_sl per wall
    wall_cos: list  # sigma cos(theta0) per wall
    wall_sg0: list  # clean solid-gas tension sigma_sg,0 per wall
    wall_sl0: list  # clean solid-liquid tension sigma_sl,0 per wall


def derive(p: OracleParams) -> Derived:
    beta = 3.0 * p.sigma / (4.0 * p.eps)
    kappa = 3.0 * p.eps * p.sigma / 8.0
    lam_s = kappa / 2.0 if p.lambda_s < 0 else p.lambda_s
    W = 4.0 * beta / p.Ex if p.Ex > 0 else 0.0
    kT = 4.0 * beta * p.Pi
    if p.phi_b > 0:
        phi_b = p.phi_b
    elif beta > 0 and p.psi_b > 0:
        phi_b = math.sqrt(1.0 - W * p.psi_b / (4.0 * beta * (1.0 - p.psi_b)))
    else:
        phi_b = 1.0
    if kappa > 0:
        M_phi = p.eta_phi * CS2 * (p.tau_g - 0.5) / kappa
    else:
        M_phi = p.M_phi
    M_0 = p.eta_psi * CS2 * (p.tau_h - 0.5) - p.M_psi * lam_s
    nu_l = CS2 * (p.tau_f - 0.5)
    nu_g = CS2 * ((p.tau_f_gas if p.tau_f_gas > 0 else p.tau_f) - 0.5)
    A, B, C, SG, SL = [], [], [], [], []
    for w in p.walls:
        c = math.cos(math.radians(w.theta0_deg))
        s_sg = p.sigma * (16.0 / 15.0 + c) / 2.0
        s_sl = p.sigma * (16.0 / 15.0 - c) / 2.0
        A.append(s_sg * w.beta_sg - s_sl * w.beta_sl)
        B.append(s_sg * w.beta_sg + s_sl * w.beta_sl)
        C.append(p.sigma * c)
        SG.append(s_sg)
        SL.append(s_sl)
    return Derived(beta, kappa, lam_s, W, kT, phi_b, M_phi, p.M_psi, M_0, nu_l, nu_g, A, B, C, SG, SL)


def clean_solid_tensions(sigma, theta0_deg):
    """sigma_sg0, sigma_sl0 from the two relations of Sec. 4.4 (Young + fixed sum 16 sigma/15)."""
    c = math.cos(math.radians(theta0_deg))
    return sigma * (16.0 / 15.0 + c) / 2.0, sigma * (16.0 / 15.0 - c) / 2.0


def psi_c_of(Ex, Pi):
    """Langmuir constant from Pi = -(1 + 2/Ex) / (4 ln psi_c)  (Sec. 4)."""
    return math.exp(-(1.0 + 2.0 / Ex) / (4.0 * Pi))
