"""FP64 CPU oracle of the learned gradient preconditioner: a 4-level U-Net
with 32 base channels, its exact backward pass, the MSE loss and Adam.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  The product
path never imports it and shares no code with it.

The paper's neural-network integration (Sec. 1 and Sec. 2.1: networks built
from the same PyTorch/JAX operations as the solvers and trained through
them) fixes no architecture.  The network here is the one the workload
names: a U-Net of 4 resolution levels (256 -> 128 -> 64 -> 32 cells per
side for a 256 x 256 input) with 32/64/128/256 channels, BF16 weights and
activations and FP32 accumulation.  Its definition (the same on both sides,
written independently on each):

  * every convolution is 3 x 3, zero padded ("same"), cross-correlation:
        y[b, h, w, co] = bias[co] + sum_{ky, kx, ci}
                         W[co, ky, kx, ci] x[b, h + ky - 1, w + kx - 1, ci]
    followed by ReLU;
  * encoder level l: two convolutions; the second one's output s_l is kept
    for the skip connection and average-pooled 2 x 2 into the next level;
  * bottleneck (level 4): two convolutions;
  * decoder level l: nearest-neighbour 2x upsampling, a convolution ("up")
    to the level's channels, concatenation [up output, s_l] along channels,
    two convolutions;
  * head: 1 x 1 convolution 32 -> 1, no activation;
  * the input has `in_ch` channels, zero-padded to 32.

Parameter layout (one flat float vector, also the layout the GPU library
takes): for each 3 x 3 layer in LAYERS order, W[cout][3][3][cin] then
bias[cout]; then the head's w[32] and bias[1].

Rounding points (where the GPU stores BF16, the oracle rounds to BF16 the
same way, FP64 -> FP32 -> BF16, round to nearest even): the padded input,
the weights (not the biases), every convolution's ReLU output, every pooled
tensor; in the backward pass every gradient of an activation (after its
ReLU mask).  Accumulations are FP64 here (FP32 on the GPU); the head output,
the loss, the weight and bias gradients and Adam are not rounded to BF16.
"""
from __future__ import annotations

import numpy as np

# (name, cin, cout) of the 3 x 3 convolutions, in parameter order
LAYERS = [
    ("enc1a", 32, 32), ("enc1b", 32, 32),
    ("enc2a", 32, 64), ("enc2b", 64, 64),
    ("enc3a", 64, 128), ("enc3b", 128, 128),
    ("bota", 128, 256), ("botb", 256, 256),
    ("up3", 256, 128), ("dec3a", 256, 128), ("dec3b", 128, 128),
    ("up2", 128, 64), ("dec2a", 128, 64), ("dec2b", 64, 64),
    ("up1", 64, 32), ("dec1a", 64, 32), ("dec1b", 32, 32),
]
IN_PAD = 32
HEAD_IN = 32


def param_count() -> int:
    n = sum(co * 9 * ci + co for _, ci, co in LAYERS)
    return n + HEAD_IN + 1


def unpack(theta):
    """Flat vector -> {name: (W[cout][3][3][cin], bias[cout])} and the head."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (param_count(),)
    out, k = {}, 0
    for name, ci, co in LAYERS:
        W = theta[k:k + co * 9 * ci].reshape(co, 3, 3, ci)
        k += co * 9 * ci
        out[name] = (W, theta[k:k + co])
        k += co
    out["head"] = (theta[k:k + HEAD_IN], theta[k + HEAD_IN:k + HEAD_IN + 1])
    return out


def pack(grads) -> np.ndarray:
    parts = []
    for name, _, _ in LAYERS:
        parts += [np.ravel(grads[name][0]), np.ravel(grads[name][1])]
    parts += [np.ravel(grads["head"][0]), np.ravel(grads["head"][1])]
    return np.concatenate(parts)


# ------------------------------------------------------------- rounding
def fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def bf16(x):
    """Round to the nearest BF16 value (ties to even) via FP32: keep the top
    16 bits of the FP32 pattern after adding 0x7FFF plus the lowest kept
    bit.  NaN stays NaN."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


# ------------------------------------------------------------ operators
def conv3x3(x, W, b):
    """Zero-padded 3 x 3 cross-correlation of x [B][H][W][ci] with
    W [co][3][3][ci], plus bias: one matrix product per tap."""
    B, H, Wd, ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((B, H, Wd, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + H, kx:kx + Wd, :] @ W[:, ky, kx, :].T
    return y


def conv3x3_backward(x, W, dy):
    """Exact transposes of conv3x3 with respect to x, W and the bias:
    dx[b, h, w, ci] = sum_{ky, kx, co} W[co, ky, kx, ci] dy[b, h - ky + 1, w - kx + 1, co],
    dW[co, ky, kx, ci] = sum_{b, h, w} dy[b, h, w, co] x[b, h + ky - 1, w + kx - 1, ci],
    db[co] = sum_{b, h, w} dy[b, h, w, co]."""
    B, H, Wd, ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            xs = xp[:, ky:ky + H, kx:kx + Wd, :]
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwi->oi", dy, xs)
            dxp[:, ky:ky + H, kx:kx + Wd, :] += dy @ W[:, ky, kx, :]
    return dxp[:, 1:-1, 1:-1], dW, dy.sum(axis=(0, 1, 2))


def avgpool2(x):
    B, H, Wd, C = x.shape
    return x.reshape(B, H // 2, 2, Wd // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dy):
    """Each input cell receives a quarter of its 2 x 2 block's gradient."""
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2)


def upsample2(x):
    """Nearest neighbour: each cell becomes a 2 x 2 block."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    """Sum over each 2 x 2 block."""
    B, H, Wd, C = dy.shape
    return dy.reshape(B, H // 2, 2, Wd // 2, 2, C).sum(axis=(2, 4))


# --------------------------------------------------------------- network
def _id(x):
    return np.asarray(x, dtype=np.float64)


def forward(theta, inp, rounding=True):
    """U-Net output [B][H][W] for input [B][H][W][in_ch]; returns (out,
    cache).  rounding=False runs the same network in plain FP64 (for the
    finite-difference pins)."""
    r = bf16 if rounding else _id
    f = fp32 if rounding else _id
    P = unpack(theta)
    Wr = {n: (r(P[n][0]), f(P[n][1])) for n, _, _ in LAYERS}
    inp = np.asarray(inp, dtype=np.float64)
    B, H, Wd, cin = inp.shape
    assert cin <= IN_PAD and H % 8 == 0 and Wd % 8 == 0
    x0 = np.zeros((B, H, Wd, IN_PAD))
    x0[..., :cin] = inp
    x0 = r(x0)
    c = {"x0": x0}

    def conv(name, x):
        y = r(np.maximum(conv3x3(x, *Wr[name]), 0.0))
        c[name] = y
        return y

    s1 = conv("enc1b", conv("enc1a", x0))
    c["p1"] = p1 = r(avgpool2(s1))
    s2 = conv("enc2b", conv("enc2a", p1))
    c["p2"] = p2 = r(avgpool2(s2))
    s3 = conv("enc3b", conv("enc3a", p2))
    c["p3"] = p3 = r(avgpool2(s3))
    bt = conv("botb", conv("bota", p3))
    c["cat3"] = cat3 = np.concatenate([conv("up3", upsample2(bt)), s3], axis=-1)
    x3 = conv("dec3b", conv("dec3a", cat3))
    c["cat2"] = cat2 = np.concatenate([conv("up2", upsample2(x3)), s2], axis=-1)
    x2 = conv("dec2b", conv("dec2a", cat2))
    c["cat1"] = cat1 = np.concatenate([conv("up1", upsample2(x2)), s1], axis=-1)
    x1 = conv("dec1b", conv("dec1a", cat1))
    wh, bh = f(P["head"][0]), f(P["head"][1])
    out = x1 @ wh + bh[0]
    c["Wr"], c["head"], c["rounding"] = Wr, (wh, bh), rounding
    return out, c


def mse(out, target):
    d = np.asarray(out, dtype=np.float64) - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d))


def backward(theta, cache, target, out):
    """Gradient of mse(out, target) with respect to the flat parameters."""
    r = bf16 if cache["rounding"] else _id
    f = fp32 if cache["rounding"] else _id
    Wr = cache["Wr"]
    wh, _ = cache["head"]
    g = {}
    N = np.asarray(out).size
    dout = f(2.0 * (np.asarray(out, dtype=np.float64) - target) / N)
    x1 = cache["dec1b"]
    g["head"] = (np.einsum("bhw,bhwc->c", dout, x1), np.array([dout.sum()]))
    dpre = r(dout[..., None] * wh * (x1 > 0))  # d (dec1b pre-activation)

    def conv_back(name, x, dpre, mask_input):
        """Weight and bias gradients of layer `name`; returns the gradient
        of its input x (times x > 0 when x is a ReLU output), rounded."""
        dx, dW, db = conv3x3_backward(x, Wr[name][0], dpre)
        g[name] = (dW, db)
        return r(dx * (x > 0)) if mask_input else r(dx)

    def decoder(level, dpre_b, x_below):
        a, cat = cache[f"dec{level}a"], cache[f"cat{level}"]
        dpre_a = conv_back(f"dec{level}b", a, dpre_b, True)
        dcat = conv_back(f"dec{level}a", cat, dpre_a, True)
        cu = Wr[f"up{level}"][0].shape[0]
        dup = conv_back(f"up{level}", upsample2(x_below), dcat[..., :cu], False)
        dx_below = r(upsample2_backward(dup) * (x_below > 0))
        return dx_below, dcat[..., cu:]

    dpre_x2, dskip1 = decoder(1, dpre, cache["dec2b"])
    dpre_x3, dskip2 = decoder(2, dpre_x2, cache["dec3b"])
    dpre_bt, dskip3 = decoder(3, dpre_x3, cache["botb"])
    dpre_ba = conv_back("botb", cache["bota"], dpre_bt, True)
    dp = conv_back("bota", cache["p3"], dpre_ba, False)
    for level, dskip in ((3, dskip3), (2, dskip2), (1, dskip1)):
        s, a = cache[f"enc{level}b"], cache[f"enc{level}a"]
        dpre_b = r(avgpool2_backward(dp) * (s > 0) + dskip)
        dpre_a = conv_back(f"enc{level}b", a, dpre_b, True)
        inp = cache[f"p{level - 1}"] if level > 1 else cache["x0"]
        if level > 1:
            dp = conv_back(f"enc{level}a", inp, dpre_a, False)
        else:
            _, dW, db = conv3x3_backward(inp, Wr["enc1a"][0], dpre_a)
            g["enc1a"] = (dW, db)
    return pack(g)


def loss_and_grad(theta, inp, target, rounding=True):
    out, cache = forward(theta, inp, rounding)
    return mse(out, target), backward(theta, cache, target, out), out


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, bias-corrected); returns new
    (theta, m, v).  `step` counts from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases; the head's
    weights with std sqrt(1 / 32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co in LAYERS:
        parts += [rng.standard_normal(co * 9 * ci) * np.sqrt(2.0 / (9 * ci)), np.zeros(co)]
    parts += [rng.standard_normal(HEAD_IN) * np.sqrt(1.0 / HEAD_IN), np.zeros(1)]
    return np.concatenate(parts)
