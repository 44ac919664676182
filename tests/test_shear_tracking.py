"""Contact-line tracking of the sheared drop: the wetted-segment finder on the wall row
(host logic), and a short sheared run on the GPU."""
import numpy as np
import pytest

from paper_2609_26332_b300.shear import wetted_segments


def test_wetted_segments_of_a_periodic_row():
    x = np.arange(64, dtype=float)
    row = np.where((x > 10.5) & (x < 20.5), 1.0, -1.0)
    row = np.tanh(np.minimum(x - 10.5, 20.5 - x))            # crossings at 10.5 and 20.5
    segs = wetted_segments(row)
    assert len(segs) == 1
    l, r = segs[0]
    assert abs(l - 10.5) < 0.05 and abs(r - 20.5) < 0.05
    # a segment across the periodic seam
    row2 = np.roll(row, 50)
    (l2, r2), = wetted_segments(row2)
    assert abs((r2 - l2) - 10.0) < 0.1 and abs(l2 - 60.5) < 0.05
    assert wetted_segments(-np.ones(8)) == [] and wetted_segments(np.ones(8)) == [(0.0, 8.0)]
    two = np.concatenate([row[:32], row[:32]])
    assert len(wetted_segments(two)) == 2


@pytest.mark.gpu
def test_sheared_drop_recedes_and_moves_downstream():
    """Under the moving top wall the wetted segment drifts downstream and narrows; with
    preferential solid-gas adsorption (beta_sg = 1) it narrows more than without
    (the dewetting trend of Sec. 4.5)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_26332_b300 import shear
    res = shear.track((0.0, 1.0), nx=256, ny=128, R=30.0, steps=6000, every=500)
    for b, r in res.items():
        print(f"beta_sg {b}: width {r['width'][0]:.3f} -> {r['width'][-1]:.3f}, "
              f"centre {r['centre'][0]:.3f} -> {r['centre'][-1]:.3f}")
        assert r["range_count"] == 0 and r["detach"] is None
        assert r["centre"][-1] > r["centre"][0]
        assert r["width"][-1] < r["width"][0]
    assert res[1.0]["width"][-1] < res[0.0]["width"][-1]
