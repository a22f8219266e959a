"""Pins of the U-Net oracle (oracle/unet.py) against what the mathematics
fixes, independent of the oracle's own code: a convolution written out as
the defining sum with explicit loops and as scipy's 2-D correlation, the
adjoint identities of every linear operator, finite differences of the whole
network's loss, torch's BF16 conversion, and Adam's closed-form first step.
Each pin is chosen so that a plausible mistake fails it; test_mutants plants
such mistakes and checks that one of the pins catches each."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import unet


def direct_conv(x, W, b):
    """The defining sum, one output value at a time (tiny inputs only)."""
    B, H, Wd, ci = x.shape
    co = W.shape[0]
    y = np.zeros((B, H, Wd, co))
    for n in range(B):
        for h in range(H):
            for w in range(Wd):
                for o in range(co):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            hh, ww = h + ky - 1, w + kx - 1
                            if 0 <= hh < H and 0 <= ww < Wd:
                                for i in range(ci):
                                    acc += W[o, ky, kx, i] * x[n, hh, ww, i]
                    y[n, h, w, o] = acc
    return y


def test_conv_equals_the_defining_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    assert np.allclose(unet.conv3x3(x, W, b), direct_conv(x, W, b), rtol=0, atol=1e-12)


def test_conv_equals_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 9, 7, 3))
    W = rng.standard_normal((2, 3, 3, 3))
    y = unet.conv3x3(x, W, np.zeros(2))
    for o in range(2):
        ref = sum(correlate2d(x[0, :, :, i], W[o, :, :, i], mode="same", boundary="fill")
                  for i in range(3))
        assert np.allclose(y[0, :, :, o], ref, atol=1e-12)


def test_conv_backward_is_the_transpose():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 6, 8, 3))
    W = rng.standard_normal((5, 3, 3, 3))
    dy = rng.standard_normal((2, 6, 8, 5))
    dx, dW, db = unet.conv3x3_backward(x, W, dy)
    # <conv(x), dy> = <x, dx> (no bias): the data adjoint
    lhs = np.sum(unet.conv3x3(x, W, np.zeros(5)) * dy)
    assert abs(lhs - np.sum(x * dx)) <= 1e-12 * abs(lhs)
    # the map W -> conv(x, W) is linear: <conv(x, dW'), dy> = <dW', dW>
    dWp = rng.standard_normal(W.shape)
    lhs = np.sum(unet.conv3x3(x, dWp, np.zeros(5)) * dy)
    assert abs(lhs - np.sum(dWp * dW)) <= 1e-12 * abs(lhs)
    assert np.allclose(db, dy.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8, 6, 3))
    y = rng.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(unet.avgpool2(x) * y), np.sum(x * unet.avgpool2_backward(y)))
    assert np.isclose(np.sum(unet.upsample2(y) * x), np.sum(y * unet.upsample2_backward(x)))
    assert np.allclose(unet.avgpool2(unet.upsample2(y)), y)
    assert np.isclose(unet.avgpool2(np.arange(4.0).reshape(1, 2, 2, 1))[0, 0, 0, 0], 1.5)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 8, 20000),
                        [0.0, -0.0, 1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9, 3.0e38, -2.5]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = unet.bf16(x)
    assert np.array_equal(got, ref)
    # ties go to the even neighbour; a value just past a tie goes up
    assert unet.bf16(1 + 2.0 ** -8) == 1.0
    assert unet.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert unet.bf16(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7


def test_param_layout():
    n = unet.param_count()
    theta = np.arange(n, dtype=np.float64)
    P = unet.unpack(theta)
    assert P["enc1a"][0].shape == (32, 3, 3, 32) and P["enc1a"][0][0, 0, 0, 0] == 0
    assert P["enc1a"][1][0] == 32 * 9 * 32
    assert np.array_equal(unet.pack(P), theta)
    assert P["head"][1][0] == n - 1
    # 17 convolutions of 3 x 3 (weights + biases, summed by hand level by
    # level) and the 1 x 1 head (32 + 1)
    assert n == (2 * 9248 + 18496 + 36928 + 73856 + 147584 + 295168 + 590080
                 + 2 * 295040 + 147584 + 2 * 73792 + 36928 + 2 * 18464 + 9248 + 33)
    assert n == 2148993


def small_net_inputs(seed, B=1, H=16, W=16):
    rng = np.random.default_rng(seed)
    theta = unet.init_params(seed)
    inp = rng.standard_normal((B, H, W, 2))
    target = rng.standard_normal((B, H, W))
    return theta, inp, target


def test_network_gradient_finite_differences():
    """Plain FP64 network (no rounding): central differences of the loss
    along random parameter directions and along single weights of several
    layers match <grad, direction> to 1e-6."""
    theta, inp, target = small_net_inputs(5)
    L, g, _ = unet.loss_and_grad(theta, inp, target, rounding=False)
    rng = np.random.default_rng(6)
    dirs = [rng.standard_normal(theta.size) * 1e-3 for _ in range(3)]
    n = 0
    for name, ci, co in unet.LAYERS:
        d = np.zeros(theta.size)
        d[n + 7 % (co * 9 * ci)] = 1e-2  # one weight
        d[n + co * 9 * ci] = 1e-2        # the first bias of the layer
        dirs.append(d)
        n += co * 9 * ci + co
    d = np.zeros(theta.size)
    d[-1] = 1e-2  # head bias
    dirs.append(d)
    for k, d in enumerate(dirs):
        # a small step: ReLU kinks make the loss only piecewise smooth, and a
        # step that moves a pre-activation across zero breaks the difference
        h = 1e-4
        Lp = unet.mse(unet.forward(theta + h * d, inp, rounding=False)[0], target)
        Lm = unet.mse(unet.forward(theta - h * d, inp, rounding=False)[0], target)
        fd = (Lp - Lm) / (2 * h)
        an = float(g @ d)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * abs(float(g @ dirs[0]))), (k, fd, an)


def test_rounded_network_stays_close_to_fp64():
    """BF16 storage moves the output by about the BF16 precision (2^-8),
    not more: the rounding points sit where the network stores tensors."""
    theta, inp, target = small_net_inputs(7)
    o64 = unet.forward(theta, inp, rounding=False)[0]
    o16 = unet.forward(theta, inp, rounding=True)[0]
    err = np.linalg.norm(o16 - o64) / np.linalg.norm(o64)
    assert 1e-5 < err < 5e-2, err


def test_adam_first_step_and_convergence():
    g = np.array([3.0, -2.0, 1e-3, 0.0])
    th, m, v = unet.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    # first bias-corrected step: m_hat = g, v_hat = g^2, so the step is
    # lr g / (|g| + eps) = lr sign(g) (and 0 for a zero gradient)
    assert np.allclose(th, [-0.1, 0.1, -0.1 * 1e-3 / (1e-3 + 1e-8), 0.0], atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # minimises a convex quadratic
    A = np.diag([1.0, 10.0, 100.0])
    x, m, v = np.array([1.0, -1.0, 2.0]), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        x, m, v = unet.adam(x, A @ x, m, v, t, lr=0.01)
    assert np.linalg.norm(x) < 1e-3


def test_mutants_are_caught(monkeypatch):
    """Plausible mistakes planted one at a time in the oracle; at least one
    pin fails for each."""
    pins = [test_conv_equals_the_defining_sum, test_conv_equals_scipy_correlation,
            test_conv_backward_is_the_transpose, test_pool_and_upsample_adjoints,
            test_network_gradient_finite_differences]
    orig = {k: getattr(unet, k) for k in ("conv3x3", "conv3x3_backward",
                                          "upsample2_backward", "avgpool2_backward")}

    def flipped_conv(x, W, b):  # convolution instead of cross-correlation
        return orig["conv3x3"](x, W[:, ::-1, ::-1, :], b)

    def unflipped_dgrad(x, W, dy):  # data gradient without the tap flip
        dx, dW, db = orig["conv3x3_backward"](x, W[:, ::-1, ::-1, :], dy)
        return dx, orig["conv3x3_backward"](x, W, dy)[1], db

    def mean_upsample_backward(dy):  # average instead of sum
        return 0.25 * orig["upsample2_backward"](dy)

    def pool_backward_no_quarter(dy):
        return 4.0 * orig["avgpool2_backward"](dy)

    def no_bias_grad(x, W, dy):
        dx, dW, db = orig["conv3x3_backward"](x, W, dy)
        return dx, dW, 0.0 * db

    mutants = [("conv3x3", flipped_conv), ("conv3x3_backward", unflipped_dgrad),
               ("upsample2_backward", mean_upsample_backward),
               ("avgpool2_backward", pool_backward_no_quarter),
               ("conv3x3_backward", no_bias_grad)]
    for name, fn in mutants:
        monkeypatch.setattr(unet, name, fn)
        failed = 0
        for pin in pins:
            try:
                pin()
            except AssertionError:
                failed += 1
        monkeypatch.setattr(unet, name, orig[name])
        assert failed > 0, name
    for pin in pins:  # and the unmodified oracle passes them all
        pin()
