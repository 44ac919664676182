"""The rest of the C-ABI boundary through the library: checkpoint/resume (slbm_save,
slbm_load) and domains living in caller-owned device memory (slbm_workspace_bytes,
slbm_create_domain_ext)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import CONFIG1, make_case, domain_for


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("precision,multiplier", [("fp32", "paper"), ("bf16", "target"), ("fp32", "exact")])
def test_save_load_resumes_bit_identically(tmp_path, precision, multiplier):
    """N steps, save, N more steps == load the file into a fresh domain, N steps: the
    fields and totals are bit-identical (the state includes the deferred multiplier
    records and the source-term history, so nothing of the next step is recomputed)."""
    _torch()
    c = make_case("ckpt", 96, 40, 0, walls=((60.0, 0.2, 0.5, 0.0), (90.0, 0.0, 0.0, 0.006)), R=12.0,
                  multiplier=multiplier)
    path = str(tmp_path / "state.slbm")
    with domain_for(c, precision=precision) as a:
        a.step(137)
        a.save(path)
        a.step(137)
        fa, ta = a.read_fields(), a.read_totals()
    assert os.path.getsize(path) > 96 * 40 * 50
    with domain_for(make_case("ckpt_other", 96, 40, 0, R=5.0, multiplier=multiplier), precision=precision) as b:
        b.set_wall(0, 60.0, 0.2, 0.5, 0.0)   # overwritten by the file's walls anyway
        b.load(path)
        assert b.read_totals()["step"] == 137
        b.step(137)
        fb, tb = b.read_fields(), b.read_totals()
    assert _same(fa, fb)
    for k in ("psi_total", "Q_phi", "H", "lambda_phi", "mubar_psi", "kinetic", "step"):
        assert ta[k] == tb[k], k


def test_load_rejects_foreign_files(tmp_path):
    torch = _torch()
    from paper_2609_26332_b300 import binding as B
    path = str(tmp_path / "a.slbm")
    with domain_for(CONFIG1) as a:
        a.step(3)
        a.save(path)
    other = make_case("other", 128, 64, 0, R=20.0, sigma=0.02)   # same grid, different sigma
    with domain_for(other) as b:
        with pytest.raises(B.SlbmError) as e:
            b.load(path)
        assert e.value.status == B.SLBM_EINVAL and "differ" in str(e.value)
        bad = str(tmp_path / "junk.slbm")
        open(bad, "wb").write(b"not a checkpoint" * 64)
        with pytest.raises(B.SlbmError):
            b.load(bad)
        trunc = str(tmp_path / "trunc.slbm")
        open(trunc, "wb").write(open(path, "rb").read()[:5000])
    with domain_for(CONFIG1) as c:
        with pytest.raises(B.SlbmError) as e:
            c.load(trunc)
        assert "truncated" in str(e.value)
        with pytest.raises(B.SlbmError):
            c.load(str(tmp_path / "missing.slbm"))


def test_domain_in_caller_workspace_allocates_nothing():
    """A domain carved from a torch-owned buffer of slbm_workspace_bytes gives the same
    fields as an ordinary domain, and creating, stepping and reading it back makes no
    device allocation (the library's own allocation count does not move)."""
    torch = _torch()
    from paper_2609_26332_b300 import binding as B
    from cases import fields0, BASE
    c = make_case("ext", 200, 72, 0, walls=((70.0, 0.3, 0.2, 0.0), (90.0, 0.0, 0.0, 0.005)), R=18.0)
    keys = [k for k in BASE if k not in ("constraint", "multiplier", "psi_on")]
    p = B.default_params(c["nx"], c["ny"], **{k: c[k] for k in keys})
    need = B.workspace_bytes(p)
    assert need > 200 * 72 * (2 * 108 + 40)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.SlbmError) as e:
        B.Domain(p, workspace=(ws.data_ptr(), need - 4096))
    assert e.value.status == B.SLBM_ENOMEM
    # the ordinary domain: the reference fields
    with domain_for(c) as r:
        r.step(60)
        fr = r.read_fields()
        tr = r.read_totals()
    # the library counts its own device allocations (the device's free memory is shared with
    # the other test processes on this GPU and moves under them)
    n0 = B.device_allocations()
    d = B.Domain(p, workspace=ws)
    for w, spec in enumerate(c["walls"]):
        d.set_wall(w, *spec)
    d.init_fields(*fields0(c))
    d.step(60)
    fe = d.read_fields()
    te = d.read_totals()
    torch.cuda.synchronize()
    assert d.device_bytes <= need
    d.close()
    assert B.device_allocations() == n0
    # the count does move for an ordinary domain
    with domain_for(c) as r2:
        r2.step(1)
    assert B.device_allocations() > n0
    assert _same(fe, fr)
    assert te["psi_total"] == tr["psi_total"]
