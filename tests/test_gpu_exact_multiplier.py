"""The exact discrete multiplier on the GPU (the constraint of Sec. 2 imposed on the
lattice field: lambda^n is the root of H(phi^{n+1}) = H(phi^0)), through the C ABI,
against the FP64 oracle's exact mode: fields element by element, the root each step
used, and the conserved measure.

Tolerances: phi, psi 1e-5 max-abs and the root 1e-4 relative, as for the paper's
multiplier.  H is held only to the FP32 arithmetic around the root, from two sources:
the per-cell terms of the cubic (and of the diagnostic sum that measures H) are FP32,
~2^-24 each and uncorrelated over N cells, and the step applies lambda through an FP32
coefficient a M_phi lambda, ~2^-24 of the multiplier's total contribution a M_phi |lambda|
sum h' <= 1.5 M_phi |lambda| N 0.75 / phi_b per step.  Neither accumulates: every step
re-targets H(phi^0).  The bound allows 8x and 4x of these."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import make_case, oracle_for, domain_for


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


U = 2.0 ** -24


def _h_tol(c, lam):
    o = oracle_for(c)
    n = c["nx"] * c["ny"]
    return 8 * np.sqrt(n) * U + 4 * U * 1.5 * o.d.M_phi * abs(lam) * n * 0.75 / o.d.phi_b


CASES = [
    # several CTAs, adsorbing bottom wall, surfactant on
    make_case("exact_drop", 96, 48, 150, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=15.0,
              multiplier="exact"),
    # ragged grid (nx not a multiple of the strip or the 16-byte chunk), moving top wall
    make_case("exact_ragged", 70, 33, 120, walls=((110.0, 0.4, 0.1, 0.0), (90.0, 0.0, 0.0, 0.005)), R=10.0,
              psi0=0.02, multiplier="exact", seed=3),
]


@pytest.mark.parametrize("c", CASES, ids=lambda c: c["name"])
def test_exact_multiplier_matches_oracle(c):
    _cuda()
    o = oracle_for(c)
    o.step(c["steps"])
    fo = o.fields()
    with domain_for(c) as d:
        H0 = d.read_totals()["H"]
        d.step(c["steps"] - 1)
        H_prev = d.read_totals()["H"]
        d.step(1)
        fg = d.read_fields()
        tg = d.read_totals()
    assert np.abs(fg["phi"] - fo["phi"]).max() < 1e-5
    assert np.abs(fg["psi"] - fo["psi"]).max() < 1e-5
    lam_o = o.log[-1]["lam"]
    assert abs(tg["lambda_phi"] - lam_o) <= 1e-4 * abs(lam_o), (tg["lambda_phi"], lam_o)
    tol = _h_tol(c, lam_o)
    for H in (H_prev, tg["H"]):
        assert abs(H - H0) <= tol, (H, H0, tol)
    assert tg["range_count"] == 0


def test_paper_multiplier_drifts_where_the_exact_one_does_not():
    _cuda()
    base = CASES[0]
    drift, lam = {}, 0.0
    for mult in ("paper", "exact"):
        c = dict(base, multiplier=mult)
        with domain_for(c) as d:
            H0 = d.read_totals()["H"]
            d.step(300)
            t = d.read_totals()
            drift[mult] = abs(t["H"] - H0)
            lam = t["lambda_phi"]
    assert drift["exact"] <= _h_tol(base, lam)
    assert drift["paper"] > 100 * max(drift["exact"], _h_tol(base, lam))


def test_linear_constraint_exact_root_is_the_mean_potential():
    """With h = phi the paper's multiplier already holds sum phi; the exact root agrees
    with the oracle's (which equals its paper value to round-off)."""
    _cuda()
    c = make_case("exact_linear", 96, 48, 100, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=15.0,
                  constraint="linear", multiplier="exact")
    o = oracle_for(c)
    o.step(c["steps"])
    with domain_for(c) as d:
        t0 = d.read_totals()
        d.step(c["steps"])
        t = d.read_totals()
        fg = d.read_fields()
    # the multiplier's total a M_phi lambda N is applied through one FP32 coefficient
    M = oracle_for(c).d.M_phi
    n = c["nx"] * c["ny"]
    assert abs(t["phi_total"] - t0["phi_total"]) <= 4 * U * 1.5 * M * abs(t["lambda_phi"]) * n + 1e-12 * abs(
        t0["phi_total"])
    assert np.abs(fg["phi"] - o.fields()["phi"]).max() < 1e-5
    lam_o = o.log[-1]["lam"]
    assert abs(t["lambda_phi"] - lam_o) <= 1e-4 * abs(lam_o)


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_exact_multiplier_in_16bit_storage(precision):
    """The root is computed from the same stored state the next step pulls, so H holds
    in the 16-bit storage modes too."""
    _cuda()
    c = CASES[0]
    with domain_for(c, precision=precision) as d:
        H0 = d.read_totals()["H"]
        d.step(200)
        t = d.read_totals()
    assert abs(t["H"] - H0) <= _h_tol(c, t["lambda_phi"])
    assert t["range_count"] == 0
