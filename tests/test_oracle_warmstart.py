"""Pins of the warm-start network oracle: the convolution against scipy's 2-D
correlation, its two adjoints and the pooling / upsampling adjoints through
inner-product identities, and the whole-network gradient against central finite
differences of the loss."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import warmstart as ws


def test_conv_is_zero_padded_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = ws.conv3x3(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = sum(correlate2d(x[n, :, :, ci], w[co, :, :, ci], mode="same", boundary="fill") for ci in range(3))
            assert np.allclose(y[n, :, :, co], ref + b[co], atol=1e-12)


def test_conv_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 10, 5))
    w = rng.standard_normal((7, 3, 3, 5))
    g = rng.standard_normal((2, 6, 10, 7))
    lhs = np.sum(ws.conv3x3(x, w) * g)
    assert np.isclose(lhs, np.sum(x * ws.conv3x3_input_grad(g, w)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(w * ws.conv3x3_weight_grad(x, g)), rtol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8, 6, 3))
    y = rng.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(ws.pool2(x) * y), np.sum(x * ws.pool2_adjoint(y)), rtol=1e-12)
    assert np.isclose(np.sum(ws.up2(y) * x), np.sum(y * ws.up2_adjoint(x)), rtol=1e-12)
    # the pool is the mean of each 2 x 2 block
    assert np.isclose(ws.pool2(x)[1, 2, 1, 0], x[1, 4:6, 2:4, 0].mean())


def _small_problem(seed=4, H=16, W=32, B=2):
    rng = np.random.default_rng(seed)
    flat = np.zeros(ws.param_count())
    layers, head = ws.unpack(flat)
    new_layers = []
    for (w, b), (_, ci, co) in zip(layers, ws.CONVS):
        new_layers.append((rng.uniform(-1, 1, w.shape) * np.sqrt(6.0 / (9 * ci)), rng.uniform(-0.1, 0.1, b.shape)))
    head = (rng.uniform(-0.4, 0.4, (2, 32)), rng.uniform(-0.1, 0.1, 2))
    flat = ws.pack(new_layers, head)
    cond = np.stack([rng.uniform([30, 0, 0, 0.005, 0.05], [150, 1, 1, 0.05, 0.09]) for _ in range(B)])
    targets = rng.standard_normal((B, 2, H, W)) * 0.5
    return flat, cond, targets


def test_network_gradient_matches_finite_differences():
    flat, cond, targets = _small_problem()
    loss, grad = ws.Net(flat).loss_grad(cond, targets)
    assert np.isclose(loss, ws.Net(flat).loss(cond, targets), rtol=1e-14)
    rng = np.random.default_rng(5)
    offs, o = [], 0
    for _, ci, co in ws.CONVS:
        offs.append((o, co * 9 * ci))          # weights of the layer
        o += co * 9 * ci
        offs.append((o, co))                   # its biases
        o += co
    offs += [(o, 64), (o + 64, 2)]             # head
    h = 1e-6
    checked = 0
    for start, count in offs:
        for k in rng.choice(count, size=min(2, count), replace=False):
            i = start + int(k)
            fp, fm = flat.copy(), flat.copy()
            fp[i] += h
            fm[i] -= h
            fd = (ws.Net(fp).loss(cond, targets) - ws.Net(fm).loss(cond, targets)) / (2 * h)
            assert abs(fd - grad[i]) <= 1e-5 * max(abs(fd), 1e-3), (i, fd, grad[i])
            checked += 1
    assert checked >= 2 * len(offs) - 2


def test_finite_differences_catch_a_planted_adjoint_error(monkeypatch):
    """A plausible slip planted in the oracle -- the upsampling adjoint averaging the
    2 x 2 children instead of summing them -- makes the gradient of a decoder weight
    disagree with the finite difference of the (unchanged) forward loss."""
    flat, cond, targets = _small_problem(seed=6)
    orig = ws.up2_adjoint
    monkeypatch.setattr(ws, "up2_adjoint", lambda g: 0.25 * orig(g))
    _, bad = ws.Net(flat).loss_grad(cond, targets)
    i = sum(co * 9 * ci + co for _, ci, co in ws.CONVS[:11]) + 7     # a weight of conv 11
    h = 1e-6
    fp, fm = flat.copy(), flat.copy()
    fp[i] += h
    fm[i] -= h
    fd = (ws.Net(fp).loss(cond, targets) - ws.Net(fm).loss(cond, targets)) / (2 * h)
    assert abs(fd) > 1e-8
    assert abs(fd - bad[i]) > 1e-3 * abs(fd)


def test_round_bf16_matches_torch_conversion():
    import torch
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        # exact ties between two BF16 values (odd and even last kept bit)
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(2.0 + 2.0 ** -7), 0.0])])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ws.round_bf16(x), ref)
