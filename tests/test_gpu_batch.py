"""Batched stepping: many instances of uneven sizes and parameters advanced by one
tile-queue launch per step (CUDA-graph replay), checked against the same instances
stepped alone and against the FP64 oracle; retirement at equilibrium; autotuner cache."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from cases import make_case, oracle_for, fields0, domain_for


def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _params_and_walls(cases, precision="fp32"):
    from paper_2609_26332_b300 import binding as B
    from cases import BASE
    keys = [k for k in BASE if k not in ("constraint", "multiplier", "psi_on")]
    params, walls = [], []
    for c in cases:
        params.append(B.default_params(c["nx"], c["ny"], precision=precision,
                                       constraint=B.LINEAR if c["constraint"] == "linear" else B.NONLINEAR,
                                       multiplier=B.TARGET if c["multiplier"] == "target" else B.PAPER,
                                       psi_on=1 if c["psi_on"] else 0, **{k: c[k] for k in keys}))
        walls.append(tuple(tuple(w) for w in c["walls"]))
    return params, walls


CASES = [
    make_case("b0", 64, 32, 0, walls=((60.0, 0.0, 0.5, 0.0), (90.0, 0.0, 0.0, 0.0)), R=10.0, seed=1),
    make_case("b1", 96, 48, 0, walls=((110.0, 0.4, 0.1, 0.0), (90.0, 0.0, 0.0, 0.005)), R=14.0, psi0=0.02, seed=2),
    make_case("b2", 70, 33, 0, walls=((45.0, 0.0, 0.9, 0.0), (90.0, 0.0, 0.0, 0.0)), R=9.0, psi0=0.03, seed=3),
    make_case("b3", 200, 100, 0, walls=((135.0, 0.9, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=30.0, seed=4),
    make_case("b4", 128, 64, 0, walls=((75.0, 0.2, 0.2, 0.0), (90.0, 0.0, 0.0, 0.0)), R=18.0,
              multiplier="target", seed=5),
    make_case("b5", 80, 40, 0, walls=((90.0, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=12.0, psi_on=False,
              seed=6),
]


def _batch(cases, band_rows=16, ctas=2, graph_steps=16, precision="fp32", width=64):
    from paper_2609_26332_b300 import binding as B
    params, walls = _params_and_walls(cases, precision)
    b = B.Batch(params, walls)
    b.set_strip_width(width)
    b.set_tiling(band_rows, ctas, graph_steps)
    for i, c in enumerate(cases):
        phi, psi = fields0(c)
        b.init_fields(i, phi, psi)
    return b


@pytest.mark.parametrize("band_rows,ctas,width", [(16, 2, 64), (64, 1, 64), (16, 3, 32), (40, 2, 32), (24, 1, 128)])
def test_batch_matches_instances_stepped_alone(band_rows, ctas, width):
    _cuda()
    steps = 100   # graph replays plus single launches
    with _batch(CASES, band_rows, ctas, graph_steps=16, width=width) as b:
        assert b.tiling() == (width, band_rows, ctas)
        b.step(steps)
        for i, c in enumerate(CASES):
            with domain_for(c) as d:
                d.step(steps)
                fs = d.read_fields()
                ts = d.read_totals()
            fb = b.read_fields(i)
            tb = b.read_totals(i)
            assert tb["step"] == steps
            for k in ("phi", "psi"):
                assert np.abs(fb[k] - fs[k]).max() < 1e-6, (c["name"], k)
            umax = max(np.abs(fs["ux"]).max(), 1e-30)
            assert np.abs(fb["ux"] - fs["ux"]).max() < 1e-4 * umax + 1e-12, c["name"]
            if c["psi_on"]:
                assert abs(tb["psi_total"] - ts["psi_total"]) <= 1e-12 * ts["psi_total"]


@pytest.mark.parametrize("width", [64, 32])
def test_batch_instances_match_oracle(width):
    _cuda()
    sel = [CASES[1], CASES[2]]
    with _batch(sel, band_rows=16, ctas=2, graph_steps=8, width=width) as b:
        b.step(150)
        for i, c in enumerate(sel):
            o = oracle_for(c)
            o.step(150)
            fo = o.fields()
            fb = b.read_fields(i)
            assert np.abs(fb["phi"] - fo["phi"]).max() < 1e-5
            assert np.abs(fb["psi"] - fo["psi"]).max() < 1e-5


def test_run_to_equilibrium_retires_converged_instances():
    _cuda()
    sel = [make_case(f"eq{k}", 64, 32, 0, walls=((60.0 + 20 * k, 0.0, 0.0, 0.0), (90.0, 0.0, 0.0, 0.0)), R=10.0,
                     psi_on=False, multiplier="target", seed=10 + k) for k in range(3)]
    with _batch(sel, band_rows=16, ctas=2, graph_steps=25) as b:
        steps = b.run_to_equilibrium(tol=1e-6, max_steps=40000, check_every=200)
        assert (steps > 0).all(), steps
        assert not b.active().any()
        before = [b.read_fields(i)["phi"] for i in range(3)]
        b.step(50)   # nothing is active: retired instances do not move
        after = [b.read_fields(i)["phi"] for i in range(3)]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)


def test_step_instance_keeps_batch_consistent():
    _cuda()
    sel = [CASES[0], CASES[2]]
    with _batch(sel, band_rows=16, ctas=2, graph_steps=8) as b:
        b.step(20)
        b.step_instance(0, 15)     # instance 0 alone
        b.step(10)
        with domain_for(sel[0]) as d:
            d.step(45)
            fs = d.read_fields()
        with domain_for(sel[1]) as d:
            d.step(30)
            f1 = d.read_fields()
        assert np.abs(b.read_fields(0)["phi"] - fs["phi"]).max() < 1e-6
        assert np.abs(b.read_fields(1)["phi"] - f1["phi"]).max() < 1e-6


def test_autotune_writes_and_reuses_cache(tmp_path):
    _cuda()
    cache = str(tmp_path / "tiling.json")
    with _batch(CASES[:3]) as b:
        br, cs = b.autotune(cache)
        w = b.tiling()[0]
        assert br in (16, 32, 64, 128, 256) and w in (32, 64, 128)
        assert 1 <= cs <= {32: 3, 64: 2, 128: 1}[w]
        data = json.load(open(cache))
        assert list(data.values()) == [[br, cs, w]]
        b.set_strip_width(32 if w != 32 else 64)    # another width, then the cached choice again
        assert b.autotune(cache) == (br, cs) and b.tiling() == (w, br, cs)
        b.step(10)
        assert b.read_totals(0)["range_count"] == 0
