"""Pins of the oracle's variable-property flow at the paper's density ratio (Sec. 4.2:
rho_l / rho_g = 1000, mu_l / mu_g = 100) with surfactant: the interpolated density and
viscosity stay within the pure-phase values although the bulk |phi| leaves phi_b(psi_b)
as the bulk surfactant adsorbs onto the interface, and the static drop stays at rest."""
import numpy as np

from oracle import Oracle, OracleParams, Wall
from paper_2609_26332_b300 import inputs


def _static_drop(steps, nx=64, ny=48):
    p = OracleParams(nx=nx, ny=ny, psi_b=0.01, rho_l=1000.0, rho_g=1.0, tau_f=0.53, tau_f_gas=0.8,
                     sigma=0.001, multiplier="target", walls=[Wall(90.0), Wall(90.0)])
    pb = inputs.bulk_phi(0.01, 1.0)
    phi0, psi0 = inputs.free_drop(nx, ny, 12.0, 4.0, phi_b=pb, psi0=0.01)
    o = Oracle(p, phi0, psi0)
    o.step(steps)
    return o


def test_density_within_phase_values_at_ratio_1000():
    o = _static_drop(200)
    e = o._evaluate()
    f = o.fields()
    raw = 0.5 * (f["phi"] / o.d.phi_b + 1.0)
    # the clip is active on both sides of the interface ...
    assert raw.min() < -1e-4 and raw.max() > 1.0 + 1e-4
    # ... and keeps rho in [rho_g, rho_l] (unclipped, rho_g + 999 chi would reach ~0.1 here)
    assert e["rho"].min() >= 1.0 and e["rho"].max() <= 1000.0
    assert 1.0 + 999.0 * raw.min() < 0.5
    # the drop stays at rest: spurious currents of the order of sigma-driven noise
    assert np.isfinite(f["ux"]).all()
    assert np.hypot(f["ux"], f["uy"]).max() < 1e-6
    tot = np.array([r["psi_total"] for r in o.log])
    assert np.abs(tot - tot[0]).max() / tot[0] < 1e-13
