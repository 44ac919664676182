"""Pins of the oracle's exact discrete multiplier (the constraint H(phi) = sum h(phi) of
Sec. 2 imposed on the discrete field): the measure is conserved to round-off, the mode
reduces to the paper's multiplier for the linear constraint (already exact there), and
its affine decomposition phi^{n+1} = A + lambda B reproduces the plain update with the
chosen lambda."""
import copy

import numpy as np

from oracle import Oracle, OracleParams, Wall
from paper_2609_26332_b300 import inputs


def _drop(multiplier, constraint="nonlinear", nx=96, ny=48):
    walls = [Wall(60.0, 0.0, 0.5, 0.0), Wall(90.0)]
    p = OracleParams(nx=nx, ny=ny, psi_b=0.01, walls=walls, multiplier=multiplier, constraint=constraint)
    phi0, psi0 = inputs.sessile_drop(nx, ny, 15.0, 4.0, phi_b=inputs.bulk_phi(0.01, 1.0), psi0=0.01,
                                     psi_noise=1e-4)
    return Oracle(p, phi0, psi0)


def test_measure_conserved_to_roundoff():
    o = _drop("exact")
    ref = _drop("paper")
    o.step(200)
    ref.step(200)
    H = np.array([r["H"] for r in o.log] + [o._H(o.fields()["phi"])])
    assert np.abs(H - o.H0).max() / o.H0 < 1e-13
    # the paper's multiplier drifts by a truncation error meanwhile
    assert abs(ref._H(ref.fields()["phi"]) - ref.H0) / ref.H0 > 1e-4
    # and the exact multiplier stays close to the paper's continuous estimate
    lam = np.array([r["lam"] for r in o.log])
    lp = np.array([r["lam_paper"] for r in o.log])
    assert np.abs(lam - lp)[50:].max() < 0.2 * np.abs(lp).max()


def test_linear_constraint_reduces_to_the_paper_multiplier():
    """With h = phi the paper's multiplier already conserves sum phi exactly on the
    lattice, so the root of the (now linear) discrete constraint is the same value."""
    o = _drop("exact", constraint="linear")
    o.step(60)
    lam = np.array([r["lam"] for r in o.log])
    lp = np.array([r["lam_paper"] for r in o.log])
    assert np.abs(lam - lp).max() <= 1e-9 * np.abs(lp).max()


def _force_lambda(o, lam):
    ev = o._evaluate

    def forced():
        e = ev()
        e["lam"] = lam
        return e
    o._evaluate = forced


def test_affine_decomposition_matches_the_plain_update():
    """Step once in exact mode; step a copy once in paper mode with lambda forced to the
    value found: the scalar populations must agree (this is where a wrong a-factor on the
    first step, a dropped w_i or a missed wall link in the B part would show)."""
    for warm in (0, 5):
        o = _drop("exact", nx=48, ny=32)
        o.step(warm)
        assert _twin_gap(o) < 1e-14


def _twin_gap(o):
    twin = copy.deepcopy(o)
    twin.p = copy.deepcopy(o.p)
    twin.p.multiplier = "paper"
    o.step(1)
    _force_lambda(twin, o.log[-1]["lam"])
    twin.step(1)
    return np.abs(o.g - twin.g).max()


def test_wrong_first_step_weight_is_caught(monkeypatch):
    """A plausible slip planted in the oracle -- the AB2 weight 1.5 given to the
    multiplier part on the first step, where R^{-1} := R^0 makes it 1 -- still conserves
    H (the root adapts to the wrong B) but no longer reproduces the plain update."""
    monkeypatch.setattr(Oracle, "_lambda_weight", lambda self: 1.5)
    o = _drop("exact", nx=48, ny=32)
    assert _twin_gap(o) > 1e-6
    assert abs(o._H(o.fields()["phi"]) - o.H0) / o.H0 < 1e-13
