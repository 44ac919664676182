"""The diagnostic totals the boundary returns beyond the conserved sums: the discrete
free energy E_f (Eq. eq1 with the wall energy of Eq. eq8) against the oracle's, the
energy law of Theorem 1 (Eq. law) on the plain-method drop run on the GPU, and the
one-step residual."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import CONFIG1, make_case, oracle_for, domain_for


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("c", [
    CONFIG1,
    make_case("energy_walls", 70, 33, 0, walls=((110.0, 0.6, 0.2, 0.0), (75.0, 0.1, 0.4, 0.0)), R=10.0, psi0=0.02),
    make_case("energy_clean", 64, 40, 0, walls=((45.0, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=12.0, psi_on=False),
], ids=["config1", "adsorbing_walls", "clean"])
def test_free_energy_matches_oracle(c):
    """E_f of the GPU diagnostic pass against Oracle.free_energy() at steps 0 and 200: the
    per-cell densities are evaluated in FP32 and summed in FP64, the fields agree to ~1e-7,
    so 2e-6 relative to |E_f| (the entropic density k_B T psi ln psi is in every cell)."""
    _cuda()
    o = oracle_for(c)
    with domain_for(c) as d:
        for n in (0, 200):
            o.step(n - o.n)
            d.step(n - d.read_totals()["step"])
            eo = o.free_energy()
            eg = d.read_totals()["free_energy"]
            assert abs(eg - eo) <= 2e-6 * abs(eo), (n, eg, eo)


def test_energy_law_on_gpu():
    """Theorem 1 (Eq. law): over the plain-method sessile drop (closed, no forcing, walls at
    rest) E_f + E_K sampled every 50 steps does not increase.  The GPU sums are FP64 of FP32
    densities, so each sample carries ~1e-7 relative noise: differences are allowed that much."""
    _cuda()
    E = []
    with domain_for(CONFIG1) as d:
        for _ in range(30):
            d.step(50)
            t = d.read_totals()
            E.append(t["free_energy"] + t["kinetic"])
    E = np.array(E)
    assert (np.diff(E) <= 2e-7 * abs(E[0])).all(), np.diff(E)
    assert E[-1] < E[0]


def test_residual_is_the_one_step_change():
    """residual = ||phi^n - phi^{n-1}||_2 / ||phi^n||_2: 0 at step 0, equal to the same
    norm of the difference of two consecutive field read-backs, and falling as the drop
    relaxes."""
    _cuda()
    with domain_for(CONFIG1) as d:
        assert d.read_totals()["residual"] < 1e-7
        d.step(99)
        a = d.read_fields(("phi",))["phi"]
        d.step(1)
        b = d.read_fields(("phi",))["phi"]
        r = d.read_totals()["residual"]
        ref = np.linalg.norm(b - a) / np.linalg.norm(b)
        # phi^{n-1} is kept in FP32 for the source terms: its rounding (~6e-8) is in r
        assert abs(r - ref) <= 2e-2 * ref + 1e-8
        d.step(2000)
        assert d.read_totals()["residual"] < r
