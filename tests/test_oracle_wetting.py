"""Pins of the oracle's wall closure against Young's law (Sec. 2.1, Eq. fw0) and the
adsorption trends of the modified Young relation (Eq. modified_young, Sec. 4.4)."""
import numpy as np
import pytest

from oracle import Oracle, OracleParams, Wall
from oracle.analysis import contact_angle
from paper_2609_26332_b300 import inputs


@pytest.mark.parametrize("theta0", [60.0, 120.0])
def test_young_angle_clean_drop(theta0):
    """Surfactant-free sessile drop, 128 x 64, R = 20, eps = 4: the wetting condition of
    Eq. boundary must give Young's angle.  The diffuse interface biases the fitted angle
    toward 90 deg (measured: 1.7 deg at 60 and 2.0 deg at 120 for R/eps = 5; 1.6 and
    0.7 deg for R/eps = 10 on 256 x 128), hence the 2.5 deg tolerance."""
    p = OracleParams(nx=128, ny=64, psi_on=False, multiplier="target", walls=[Wall(theta0), Wall(90.0)])
    phi0, _ = inputs.sessile_drop(128, 64, 20.0, 4.0)
    o = Oracle(p, phi0)
    o.step(4000)
    th, _ = contact_angle(o.fields()["phi"], 4.0)
    assert abs(th - theta0) < 2.5


def test_solid_adsorption_trends():
    """Sec. 4.4: preferential solid-liquid adsorption (beta_sl > beta_sg) lowers the
    angle (hydrophilisation), preferential solid-gas adsorption raises it (autophobing),
    relative to the same surfactant-laden drop without solid adsorption."""
    ang = {}
    for name, (bsg, bsl) in {"none": (0.0, 0.0), "sl": (0.01, 0.9), "sg": (0.9, 0.01)}.items():
        p = OracleParams(nx=128, ny=64, psi_b=0.02, multiplier="target",
                         walls=[Wall(90.0, bsg, bsl, 0.0), Wall(90.0)])
        phi0, psi0 = inputs.sessile_drop(128, 64, 20.0, 4.0, phi_b=inputs.bulk_phi(0.02, 1.0), psi0=0.02)
        o = Oracle(p, phi0, psi0)
        o.step(3000)
        ang[name], _ = contact_angle(o.fields()["phi"], 4.0)
    assert ang["sl"] < ang["none"] - 1.0
    assert ang["sg"] > ang["none"] + 1.0
