"""The two input stagings of the step kernel (slbm_params.staging): TMA tile copies with
mbarriers against thread-issued cp.async, in every storage mode, with the exact
multiplier, at the periodic seam and across several strips.  They move the same values,
but they are separate kernel instantiations (and the FP32 cp.async one loads the
collide's inputs earlier), and the compiler chooses for each where plain FP32 expressions
become fused multiply-adds: the fields agree to rounding, not bitwise.  A wrong staged
value (a halo column, a seam image, a stale row) changes phi and psi by 1e-2 or more
within a few steps; after 3 steps the fields are compared to 5e-7 (FP32) and 1e-3 (16-bit
storage, a few units in the last place of a population), after 300 steps to 1e-5 and
1e-3 (measured: FP32 at most a few 1e-8; FP16 6e-5 after a one-rounding difference of the
surfactant multiplier near step 20).  The TMA path is also checked against the oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import make_case, oracle_for, domain_for


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(c, precision, staging, steps):
    with domain_for(c, precision=precision, staging=staging) as d:
        d.step(steps)
        return d.read_fields(), d.read_totals()


@pytest.mark.parametrize("precision,multiplier", [("fp32", "paper"), ("fp16", "target"), ("bf16", "paper"),
                                                  ("fp32", "exact")])
def test_tma_and_cpasync_staging_agree(precision, multiplier):
    _cuda()
    # 256 x 96: four strips (two at the seam), a moving top wall, adsorbing bottom wall
    c = make_case("staging", 256, 96, 0, walls=((70.0, 0.3, 0.6, 0.0), (90.0, 0.0, 0.0, 0.008)), R=20.0,
                  multiplier=multiplier)
    fa, ta = _run(c, precision, 0, 3)
    fb, tb = _run(c, precision, 1, 3)
    tol = 5e-7 if precision == "fp32" else 1e-3
    for k in fa:
        assert np.abs(fa[k] - fb[k]).max() <= tol, k
    assert abs(ta["psi_total"] - tb["psi_total"]) <= 1e-12 * ta["psi_total"]
    for k, rel in (("H", 1e-6), ("free_energy", 1e-6), ("kinetic", 1e-5)):
        assert abs(ta[k] - tb[k]) <= rel * abs(ta[k]), k
    fa, ta = _run(c, precision, 0, 300)
    fb, tb = _run(c, precision, 1, 300)
    tol = 1e-5 if precision == "fp32" else 1e-3
    for k in fa:
        assert np.abs(fa[k] - fb[k]).max() <= tol, k
    assert abs(ta["psi_total"] - tb["psi_total"]) <= 1e-12 * ta["psi_total"]
    assert abs(ta["free_energy"] - tb["free_energy"]) <= 1e-6 * abs(ta["free_energy"])


def test_tma_staging_against_the_oracle():
    _cuda()
    c = make_case("staging_oracle", 128, 48, 400, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.005)), R=14.0)
    o = oracle_for(c)
    o.step(c["steps"])
    fo = o.fields()
    fg, tg = _run(c, "fp32", 1, c["steps"])
    assert np.abs(fg["phi"] - fo["phi"]).max() < 1e-5
    assert np.abs(fg["psi"] - fo["psi"]).max() < 1e-5
    umax = max(np.abs(fo["ux"]).max(), np.abs(fo["uy"]).max())
    assert max(np.abs(fg["ux"] - fo["ux"]).max(), np.abs(fg["uy"] - fo["uy"]).max()) <= 1e-5 * umax + 2e-8
    assert abs(tg["psi_total"] - o.totals()["psi_total"]) <= 1e-12 * tg["psi_total"]
