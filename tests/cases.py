"""Seeded parity cases: one plain description turned into oracle parameters, library
parameters and initial fields (test harness only; the two sides share nothing else)."""
import numpy as np

from oracle import Oracle, OracleParams, Wall
from paper_2609_26332_b300 import inputs

BASE = dict(tau_f=0.8, tau_f_gas=-1.0, tau_g=0.8, tau_h=0.8, sigma=0.01, eps=4.0, Ex=1.0, Pi=0.18407,
            M_phi=0.0, M_psi=0.5, eta_phi=1.0, eta_psi=1.0, lambda_s=-1.0, psi_b=0.0, phi_b=-1.0,
            rho_l=1.0, rho_g=1.0, Gx=0.0, Gy=0.0, constraint="nonlinear", multiplier="paper", psi_on=True,
            mrt_f=(0.0, 0.0, 0.0, 0.0), mrt_g=(0.0, 0.0, 0.0, 0.0), mrt_h=(0.0, 0.0, 0.0, 0.0))


def make_case(name, nx, ny, steps, walls=((90.0, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), init="sessile",
              R=None, psi0=0.01, psi_noise=1e-4, seed=inputs.DEFAULT_SEED, **kw):
    c = dict(BASE)
    c.update(kw)
    c.update(name=name, nx=nx, ny=ny, steps=steps, walls=walls, init=init, R=R, psi0=psi0,
             psi_noise=psi_noise, seed=seed)
    if c["psi_on"] and c["psi_b"] == 0.0:
        c["psi_b"] = psi0
    return c


def fields0(c):
    nx, ny = c["nx"], c["ny"]
    R = c["R"] if c["R"] is not None else 0.3 * ny
    pb = inputs.bulk_phi(c["psi_b"] if c["psi_on"] else 0.0, c["Ex"])
    psi0 = c["psi0"] if c["psi_on"] else 0.0
    if c["init"] == "sessile":
        phi, psi = inputs.sessile_drop(nx, ny, R, c["eps"], phi_b=pb, psi0=psi0,
                                       psi_noise=c["psi_noise"] if c["psi_on"] else 0.0, seed=c["seed"])
    elif c["init"] == "free":
        phi, psi = inputs.free_drop(nx, ny, R, c["eps"], phi_b=pb, psi0=psi0)
    elif c["init"] == "drops":
        phi, _ = inputs.drop_field(nx, ny, c.get("n_drops", 4), 0.12 * ny, 0.2 * ny, c["eps"], 2 * c["eps"],
                                   seed=c["seed"], phi_b=pb)
        psi = np.full((ny, nx), psi0)
    else:
        raise ValueError(c["init"])
    return phi, (psi if c["psi_on"] else None)


def oracle_for(c):
    keys = [k for k in BASE if k not in ("constraint", "multiplier", "psi_on")]
    p = OracleParams(nx=c["nx"], ny=c["ny"], constraint=c["constraint"], multiplier=c["multiplier"],
                     psi_on=c["psi_on"], walls=[Wall(*c["walls"][0]), Wall(*c["walls"][1])],
                     **{k: c[k] for k in keys})
    phi, psi = fields0(c)
    return Oracle(p, phi, psi)


def domain_for(c, precision="fp32", stream=None, staging=0):
    from paper_2609_26332_b300 import binding as B
    keys = [k for k in BASE if k not in ("constraint", "multiplier", "psi_on")]
    p = B.default_params(c["nx"], c["ny"], precision=precision, staging=staging,
                         constraint=B.LINEAR if c["constraint"] == "linear" else B.NONLINEAR,
                         multiplier={"paper": B.PAPER, "target": B.TARGET, "exact": B.EXACT}[c["multiplier"]],
                         psi_on=1 if c["psi_on"] else 0, **{k: c[k] for k in keys})
    d = B.Domain(p, stream=stream)
    for w, spec in enumerate(c["walls"]):
        d.set_wall(w, *spec)
    phi, psi = fields0(c)
    d.init_fields(phi, psi)
    return d


# the plain-method sessile drop (128 x 64, R = 20, eps = 4, tau = 0.8, 60 deg,
# psi0 = 0.01 +- 1e-4, solid-liquid adsorption 0.5)
CONFIG1 = make_case("config1", 128, 64, 1000, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=20.0)
