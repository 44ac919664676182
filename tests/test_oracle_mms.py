"""Manufactured-solution convergence of the scalar lattice Boltzmann equations (Sec. 4.1,
accuracy test): second order in space under diffusive scaling for phi and psi, the
globally conserved sums held to round-off, and the printed closed form of the mean
surfactant potential checked by quadrature."""
import math

import numpy as np
import pytest

from oracle import mms


def test_mean_surfactant_potential_closed_form():
    n = 256
    c = np.arange(n) / n
    x, y = np.meshgrid(c, c)
    for t in (0.0, 0.7, 3.0):
        pe, qe = mms.exact(x, y, t)
        assert abs(mms.mu_psi_bulk(pe, qe).mean() - mms.mubar_psi_exact(t)) < 1e-12
        # and the phi potential averages to zero (sin * cos modes)
        assert abs((mms.mu_phi_bulk(pe, qe) + mms.KAPPA * 8 * math.pi ** 2 * pe).mean()) < 1e-12


def test_second_order_convergence_and_conservation():
    res = {n: mms.run(n) for n in (16, 32, 64)}
    for a, b in ((16, 32), (32, 64)):
        o_phi = math.log2(res[a][0] / res[b][0])
        o_psi = math.log2(res[a][1] / res[b][1])
        print(f"dx 1/{a} -> 1/{b}: order phi {o_phi:.3f}, psi {o_psi:.3f}")
        assert 1.9 < o_phi < 2.1 and 1.9 < o_psi < 2.1
    for n, r in res.items():
        assert r[3] < 1e-12 and r[4] < 1e-13, (n, r[3], r[4])


def test_a_wrong_mean_potential_is_caught(monkeypatch):
    """A plausible slip planted in the oracle -- the sign of the adsorption term of the
    closed-form mean potential flipped -- gives the psi source a nonzero mean, which the
    mass constraint cannot absorb: sum psi drifts by ~1e-4 instead of round-off, and the
    psi error grows."""
    good = mms.run(32, t_end=1.0)
    orig = mms.mubar_psi_exact
    monkeypatch.setattr(mms, "mubar_psi_exact",
                        lambda t: orig(t) - 2 * mms.WADS * (mms.AMP * math.exp(-t)) ** 2 / 8.0)
    bad = mms.run(32, t_end=1.0)
    assert good[4] < 1e-13 and bad[4] > 5e-5
    assert bad[1] > 1.02 * good[1]


def test_channel_form_second_order_and_conservation():
    """The channel form of the test (u = (0.05, 0), both fields varying as cos 2 pi y so
    that the neutral walls' zero-flux closure is exact for them), run through the full
    Oracle with a prescribed velocity and the manufactured sources: second order in space
    for phi and psi, sum psi to round-off."""
    res = {n: mms.run_channel(n) for n in (16, 32, 64)}
    for a, b in ((16, 32), (32, 64)):
        o_phi = math.log2(res[a][0] / res[b][0])
        o_psi = math.log2(res[a][1] / res[b][1])
        print(f"channel dx 1/{a} -> 1/{b}: order phi {o_phi:.3f}, psi {o_psi:.3f}")
        assert 1.9 < o_phi < 2.1 and 1.9 < o_psi < 2.1
    for n, r in res.items():
        assert r[3] < 1e-12, (n, r[3])
