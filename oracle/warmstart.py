"""FP64 CPU oracle of the warm-start network (test infrastructure only).

The paper has no network: this is the definition of the convolutional encoder-decoder
the library trains to predict relaxed sessile-drop states, written out plainly in
numpy float64 so that the tensor-core forward, input-gradient and weight-gradient
kernels and the whole-network gradient can be checked against it.

* ``conv3x3`` / ``conv3x3_input_grad`` / ``conv3x3_weight_grad`` - the 3 x 3, stride-1,
  zero-padded convolution of NHWC tensors with weights w[co][ky][kx][ci] (tap (ky, kx)
  multiplies x[y + ky - 1][x + kx - 1]) and its two adjoints, one tap at a time.
* ``features`` - the 16 input channels built from a parameter row (theta0 [deg],
  beta_sg, beta_sl, psi0, area fraction) and the cell coordinates.
* ``Net`` - the architecture (4 levels of two convs, 2 x 2 average pooling, nearest
  upsampling with skip concatenation, a 1 x 1 head), its loss and the gradient of the
  loss by reverse-mode differentiation written out layer by layer.  An optional
  rounding ``q`` (``round_bf16``) is applied wherever the GPU stores a tensor in BF16,
  so that both sides take the same rounding decisions.

Pins: ``tests/test_oracle_warmstart.py`` ties the convolution to scipy's 2-D
correlation, the adjoints to the forward through inner-product identities, the
whole-network gradient to central finite differences of the loss, and ``round_bf16``
to torch's float32 -> bfloat16 conversion.
"""

import numpy as np

CONVS = [(0, 16, 32), (0, 32, 32), (1, 32, 64), (1, 64, 64), (2, 64, 128), (2, 128, 128), (3, 128, 128),
         (3, 128, 128), (2, 256, 128), (2, 128, 128), (1, 192, 64), (1, 64, 64), (0, 96, 32), (0, 32, 32)]
HEAD = 32


def _shift(x, dy, dx):
    """s[b, y, x] = x[b, y + dy, x + dx] with zeros outside the image."""
    B, H, W, C = x.shape
    s = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    if ys < ye and xs < xe:
        s[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return s


def conv3x3(x, w, b=None):
    """y[b, y, x, co] = b[co] + sum_{ky, kx, ci} x[b, y + ky - 1, x + kx - 1, ci] w[co, ky, kx, ci]."""
    B, H, W, _ = x.shape
    y = np.zeros((B, H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += _shift(x, ky - 1, kx - 1) @ w[:, ky, kx, :].T
    if b is not None:
        y += b
    return y


def conv3x3_input_grad(g, w):
    """Adjoint of x -> conv3x3(x, w): dx[b, y, x, ci] = sum g[b, y - ky + 1, x - kx + 1, co] w[co, ky, kx, ci]."""
    dx = np.zeros(g.shape[:3] + (w.shape[3],))
    for ky in range(3):
        for kx in range(3):
            dx += _shift(g, 1 - ky, 1 - kx) @ w[:, ky, kx, :]
    return dx


def conv3x3_weight_grad(x, g):
    """Adjoint of w -> conv3x3(x, w): dw[co, ky, kx, ci] = sum_{b, y, x} g[b, y, x, co] x[b, y + ky - 1, x + kx - 1, ci]."""
    Co, Ci = g.shape[3], x.shape[3]
    dw = np.zeros((Co, 3, 3, Ci))
    g2 = g.reshape(-1, Co)
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = g2.T @ _shift(x, ky - 1, kx - 1).reshape(-1, Ci)
    return dw


def pool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_adjoint(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_adjoint(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def features(cond, H, W):
    """Input channels [B, H, W, 16] of parameter rows cond [B, 5]."""
    cond = np.asarray(cond, dtype=np.float64)
    B = cond.shape[0]
    half = 0.5 * H
    X = (np.arange(W) + 0.5 - 0.5 * W) / half
    Y = (np.arange(H) + 0.5) / half
    Xg, Yg = np.meshgrid(X, Y)
    f = np.zeros((B, H, W, 16))
    for b in range(B):
        c = cond[b]
        f[b, :, :, 0] = (c[0] - 90.0) / 60.0
        f[b, :, :, 1] = 2.0 * c[1] - 1.0
        f[b, :, :, 2] = 2.0 * c[2] - 1.0
        f[b, :, :, 3] = (c[3] - 0.0275) / 0.0225
        f[b, :, :, 4] = (c[4] - 0.07) / 0.025
        f[b, :, :, 5] = Xg
        f[b, :, :, 6] = Yg
        f[b, :, :, 7] = 1.0
        f[b, :, :, 8] = Xg * Xg
        f[b, :, :, 9] = Yg * Yg
        f[b, :, :, 10] = Xg * Yg
        f[b, :, :, 11] = np.abs(Xg)
        f[b, :, :, 12] = np.sin(0.5 * np.pi * Xg)
        f[b, :, :, 13] = np.cos(0.5 * np.pi * Xg)
        f[b, :, :, 14] = np.sin(0.5 * np.pi * Yg)
        f[b, :, :, 15] = np.cos(0.5 * np.pi * Yg)
    return f


def unpack(flat):
    """Flat parameter vector (library order) -> list of (w [Co,3,3,Ci], b [Co]) and head (w [2,32], b [2])."""
    flat = np.asarray(flat, dtype=np.float64)
    layers, o = [], 0
    for _, ci, co in CONVS:
        w = flat[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
        o += co * 9 * ci
        b = flat[o:o + co]
        o += co
        layers.append((w, b))
    hw = flat[o:o + 2 * HEAD].reshape(2, HEAD)
    o += 2 * HEAD
    hb = flat[o:o + 2]
    o += 2
    assert o == flat.size, "parameter count mismatch"
    return layers, (hw, hb)


def pack(layers, head):
    parts = []
    for w, b in layers:
        parts += [w.ravel(), b.ravel()]
    parts += [head[0].ravel(), head[1].ravel()]
    return np.concatenate(parts)


def param_count():
    return sum(co * 9 * ci + co for _, ci, co in CONVS) + 2 * HEAD + 2


class Net:
    """The encoder-decoder with parameters ``flat`` (library order)."""

    def __init__(self, flat):
        self.layers, self.head = unpack(flat)

    def forward(self, cond, H, W, q=None):
        """Head outputs [B, 2, H, W] and the activations the backward pass needs.

        q: optional rounding applied to every stored activation (the input features,
        each conv output, each pooled tensor); None = exact FP64."""
        q = q or (lambda t: t)
        L = self.layers
        relu = lambda z: np.maximum(z, 0.0)
        conv = lambda x, i: q(relu(conv3x3(x, *L[i])))
        a = {}
        a["x0"] = q(features(cond, H, W))
        a["y0"] = conv(a["x0"], 0)
        a["y1"] = conv(a["y0"], 1)
        a["p0"] = q(pool2(a["y1"]))
        a["y2"] = conv(a["p0"], 2)
        a["y3"] = conv(a["y2"], 3)
        a["p1"] = q(pool2(a["y3"]))
        a["y4"] = conv(a["p1"], 4)
        a["y5"] = conv(a["y4"], 5)
        a["p2"] = q(pool2(a["y5"]))
        a["y6"] = conv(a["p2"], 6)
        a["y7"] = conv(a["y6"], 7)
        a["c2"] = np.concatenate([up2(a["y7"]), a["y5"]], axis=3)
        a["y8"] = conv(a["c2"], 8)
        a["y9"] = conv(a["y8"], 9)
        a["c1"] = np.concatenate([up2(a["y9"]), a["y3"]], axis=3)
        a["y10"] = conv(a["c1"], 10)
        a["y11"] = conv(a["y10"], 11)
        a["c0"] = np.concatenate([up2(a["y11"]), a["y1"]], axis=3)
        a["y12"] = conv(a["c0"], 12)
        a["y13"] = conv(a["y12"], 13)
        hw, hb = self.head
        out = a["y13"] @ hw.T + hb                      # [B, H, W, 2]
        return np.moveaxis(out, 3, 1), a

    def loss(self, cond, targets):
        """Mean over cells of the squared errors of both output channels (summed)."""
        targets = np.asarray(targets, dtype=np.float64)
        out, _ = self.forward(cond, targets.shape[2], targets.shape[3])
        B, _, H, W = targets.shape
        return float(((out - targets) ** 2).sum() / (B * H * W))

    def loss_grad(self, cond, targets, q=None):
        """(loss, flat gradient) by reverse-mode differentiation.

        gz[i] is the gradient w.r.t. the pre-activation output of conv i (the ReLU mask
        applied); the weight and bias gradients of conv i follow from gz[i] and the
        conv's input.  q: optional rounding of every stored activation and of every
        stored gradient tensor (gz[i], the gradients w.r.t. the concatenated and pooled
        conv inputs); None = exact FP64."""
        q = q or (lambda t: t)
        targets = np.asarray(targets, dtype=np.float64)
        B, _, H, W = targets.shape
        out, a = self.forward(cond, H, W, q)
        n = B * H * W
        r = out - targets
        loss = float((r ** 2).sum() / n)
        go = np.moveaxis(2.0 * r / n, 1, 3)             # d loss / d head output, [B, H, W, 2]
        hw, hb = self.head
        g_hw = go.reshape(-1, 2).T @ a["y13"].reshape(-1, HEAD)
        g_hb = go.reshape(-1, 2).sum(axis=0)
        L = self.layers
        on = lambda name: a[name] > 0                   # ReLU mask of a stored activation
        back = lambda i, g: conv3x3_input_grad(g, L[i][0])
        gz = [None] * len(L)
        gz[13] = q((go @ hw) * on("y13"))
        gz[12] = q(back(13, gz[13]) * on("y12"))
        g_c0 = q(back(12, gz[12]) * on("c0"))           # w.r.t. the concatenation (up(y11), y1)
        gz[11] = q(up2_adjoint(g_c0[..., :64]) * on("y11"))
        gz[10] = q(back(11, gz[11]) * on("y10"))
        g_c1 = q(back(10, gz[10]) * on("c1"))           # (up(y9), y3)
        gz[9] = q(up2_adjoint(g_c1[..., :128]) * on("y9"))
        gz[8] = q(back(9, gz[9]) * on("y8"))
        g_c2 = q(back(8, gz[8]) * on("c2"))             # (up(y7), y5)
        gz[7] = q(up2_adjoint(g_c2[..., :128]) * on("y7"))
        gz[6] = q(back(7, gz[7]) * on("y6"))
        g_p2 = q(back(6, gz[6]))                        # w.r.t. the pooled p2 (no ReLU there)
        gz[5] = q((pool2_adjoint(g_p2) + g_c2[..., 128:]) * on("y5"))
        gz[4] = q(back(5, gz[5]) * on("y4"))
        g_p1 = q(back(4, gz[4]))
        gz[3] = q((pool2_adjoint(g_p1) + g_c1[..., 128:]) * on("y3"))
        gz[2] = q(back(3, gz[3]) * on("y2"))
        g_p0 = q(back(2, gz[2]))
        gz[1] = q((pool2_adjoint(g_p0) + g_c0[..., 64:]) * on("y1"))
        gz[0] = q(back(1, gz[1]) * on("y0"))
        inputs = ["x0", "y0", "p0", "y2", "p1", "y4", "p2", "y6", "c2", "y8", "c1", "y10", "c0", "y12"]
        gw = [conv3x3_weight_grad(a[inputs[i]], gz[i]) for i in range(len(L))]
        gb = [gz[i].reshape(-1, gz[i].shape[3]).sum(axis=0) for i in range(len(L))]
        return loss, pack(list(zip(gw, gb)), (g_hw, g_hb))


def round_bf16(x):
    """x rounded to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)
