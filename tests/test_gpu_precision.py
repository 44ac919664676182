"""Precision modes: populations and history stored in FP16 / BF16 as deviations from the
rest equilibrium, collisions in FP32, zeroth moments in float-float, integrals in FP64.

Checked against the FP64 oracle on the same seeded inputs:
* conserved totals within 1e-10 relative (the bookkeeping does not depend on storage);
* the equilibrium contact angle within 0.5 deg of the oracle's;
* per-field errors after 1000 steps are reported (printed) and bounded loosely
  (FP16 keeps 11 significant bits of each stored deviation, BF16 8 bits).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import CONFIG1, make_case, oracle_for, domain_for
from oracle.analysis import contact_angle


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def oracle_1000():
    o = oracle_for(CONFIG1)
    o.step(1000)
    return o.fields(), o.totals()


@pytest.mark.parametrize("prec,bound", [("fp32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-2)])
def test_fields_and_totals_after_1000_steps(prec, bound, oracle_1000):
    _cuda()
    fo, to = oracle_1000
    with domain_for(CONFIG1, precision=prec) as d:
        d.step(1000)
        fg = d.read_fields()
        tg = d.read_totals()
    err = {k: float(np.abs(fg[k] - fo[k]).max()) for k in ("phi", "psi")}
    umax = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max())
    err["u_rel"] = float(max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max()) / umax)
    err["psi_total_rel"] = abs(tg["psi_total"] - to["psi_total"]) / to["psi_total"]
    print(f"{prec}: per-field max error after 1000 steps {err}")
    assert err["psi_total_rel"] < 1e-10
    assert err["phi"] < bound and err["psi"] < bound
    assert tg["range_count"] == 0 and tg["clamp_count"] == 0


@pytest.fixture(scope="module")
def oracle_equilibrium():
    c = make_case("angle", 128, 64, 5000, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=20.0,
                  multiplier="target")
    o = oracle_for(c)
    o.step(c["steps"])
    th, _ = contact_angle(o.fields()["phi"], c["eps"])
    return c, th, o.totals()


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_equilibrium_angle_matches_oracle(prec, oracle_equilibrium):
    """Surfactant-laden sessile drop (60 deg, solid-liquid adsorption 0.5) relaxed for 5000
    steps: the GPU angle in each storage mode within 0.5 deg of the FP64 oracle's."""
    _cuda()
    c, th_o, to = oracle_equilibrium
    with domain_for(c, precision=prec) as d:
        d.step(c["steps"])
        th_g, _ = contact_angle(d.read_fields()["phi"], c["eps"])
        tg = d.read_totals()
    print(f"{prec}: angle {th_g:.3f} vs oracle {th_o:.3f}; "
          f"sum psi rel diff {abs(tg['psi_total'] - to['psi_total']) / to['psi_total']:.2e}")
    assert abs(th_g - th_o) < 0.5
    assert abs(tg["psi_total"] - to["psi_total"]) / to["psi_total"] < 1e-10
