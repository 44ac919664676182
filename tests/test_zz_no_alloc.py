"""slbm_read_fields_noalloc: the fields and totals of the current time level written into
buffers the caller owns, with the reduction scratch in the library's static device array
instead of any allocation.  Some callers cannot allocate device memory once they run (a
host framework or pool owns and budgets it all); this entry point serves them.  Its output
must match the allocating slbm_read_fields / slbm_read_totals, on two calls in a row."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import make_case, domain_for


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_matches_allocating_readout_twice():
    torch = _torch()
    c = make_case("noalloc", 96, 48, 0, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.004)), R=14.0)
    with domain_for(c) as d:
        bufs = {k: torch.empty((48, 96), dtype=torch.float64, device="cuda")
                for k in ("phi", "psi", "ux", "uy", "p")}
        for n in (25, 40):
            d.step(n)
            ref = d.read_fields()
            tref = d.read_totals()
            for call in range(2):            # two calls in a row share the static scratch
                for b in bufs.values():
                    b.fill_(float("nan"))
                t = d.read_fields_noalloc(**bufs)
                torch.cuda.synchronize()
                for k in bufs:
                    got = bufs[k].cpu().numpy()
                    assert np.isfinite(got).all()
                    scale = max(np.abs(ref[k]).max(), 1e-30)
                    assert np.abs(got - ref[k]).max() <= 1e-12 * scale, (k, call)
                for k in ("psi_total", "Q_phi", "H", "lambda_phi", "mubar_psi", "kinetic"):
                    assert abs(t[k] - tref[k]) <= 1e-12 * max(abs(tref[k]), 1e-30), (k, call)
                assert t["step"] == tref["step"] and t["range_count"] == 0
        # a subset of outputs and no totals: queues work only
        assert d.read_fields_noalloc(phi=bufs["phi"], totals=False) is None
        torch.cuda.synchronize()
        assert np.abs(bufs["phi"].cpu().numpy() - d.read_fields()["phi"]).max() <= 1e-12
