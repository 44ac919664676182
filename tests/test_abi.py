"""CPU checks of the C-ABI library: it loads, exports every function declared in
include/surflbm.h, and rejects bad parameters before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(slbm(?:3d)?_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2609_26332_b300 import binding as B
    names = _declared()
    assert "slbm_step" in names and "slbm_create_domain" in names and "slbm3d_step" in names
    for n in names:
        assert hasattr(B.lib, n), n
    assert "sm_103a" in B.version()


def test_default_params_and_validation():
    from paper_2609_26332_b300 import binding as B
    p = B.default_params(128, 64)
    assert p.nx == 128 and p.ny == 64 and abs(p.tau_f - 0.8) < 1e-15 and p.psi_on == 1
    for bad in (dict(ny=1), dict(tau_f=0.5), dict(eps=0.0), dict(psi_b=1.0), dict(precision=7),
                dict(mrt_f=(0, 2.5, 0, 0)), dict(rho_g=-1.0), dict(constraint=3), dict(multiplier=3),
                dict(nx=1 << 15, ny=1 << 14), dict(nx=0)):
        q = B.default_params(64, 32)
        for k, v in bad.items():
            if k in ("mrt_f",):
                for j, x in enumerate(v):
                    q.mrt_f[j] = x
            else:
                setattr(q, k, v)
        with pytest.raises(B.SlbmError) as e:
            B.Domain(q)
        assert e.value.status == B.SLBM_EINVAL
    # the exact multiplier is a single-domain mode: a batch refuses it before any allocation
    ok, ex = B.default_params(64, 32), B.default_params(64, 32, multiplier=B.EXACT)
    with pytest.raises(B.SlbmError) as e:
        B.Batch([ok, ex])
    assert e.value.status == B.SLBM_EINVAL and "single domains" in str(e.value)
    # NULL handles are rejected without a crash
    assert B.lib.slbm_step(None, 1) == B.SLBM_EINVAL
    assert B.lib.slbm_set_walls(None, 0, 90.0, 0.0, 0.0, 0.0) == B.SLBM_EINVAL
    B.lib.slbm_destroy(None)


def test_warm_start_entry_points_validate_before_touching_the_gpu():
    import ctypes
    from paper_2609_26332_b300 import binding as B
    h = ctypes.c_void_p()
    for ny, nx, mb in ((12, 32, 1), (16, 30, 1), (16, 32, 0)):
        assert B.lib.slbm_ws_create(ny, nx, mb, 1, None, ctypes.byref(h)) == B.SLBM_EINVAL
    # channel counts the tensor-core tiles cannot take
    assert B.lib.slbm_conv3x3_forward(None, None, None, None, 1, 8, 8, 16, 32, 1, None) == B.SLBM_EINVAL
    fake = ctypes.c_void_p(1 << 20)
    assert B.lib.slbm_conv3x3_forward(fake, fake, None, fake, 1, 8, 8, 12, 32, 1, None) == B.SLBM_EINVAL
    assert B.lib.slbm_conv3x3_forward(fake, fake, None, fake, 1, 8, 8, 16, 40, 1, None) == B.SLBM_EINVAL
    assert B.lib.slbm_conv3x3_input_grad(fake, fake, None, fake, 1, 8, 8, 24, 32, None) == B.SLBM_EINVAL
    assert B.lib.slbm_conv3x3_weight_grad(fake, fake, fake, 1, 8, 8, 32, 256, None) == B.SLBM_EINVAL
    assert B.lib.slbm_ws_param_count(None) == 0


def test_3d_extension_rejects_what_it_does_not_cover():
    """The three-dimensional domain refuses, before touching the GPU, the modes it does not
    implement: 16-bit storage, MRT rates, variable density, the exact multiplier, nz < 1."""
    from paper_2609_26332_b300 import binding as B
    for bad in (dict(precision=B._PREC["bf16"]), dict(rho_l=10.0), dict(multiplier=B.EXACT), dict(tau_f_gas=0.6)):
        q = B.default_params(16, 8, **bad)
        with pytest.raises(B.SlbmError) as e:
            B.Domain3D(q, 8)
        assert e.value.status == B.SLBM_EINVAL
    q = B.default_params(16, 8, mrt_g=(0.0, 1.2, 0.0, 0.0))
    with pytest.raises(B.SlbmError):
        B.Domain3D(q, 8)
    with pytest.raises(B.SlbmError):
        B.Domain3D(B.default_params(16, 8), 0)
