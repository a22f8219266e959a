"""Parity of the U-Net preconditioner's CUDA path (tcgen05 convolutions,
element-wise kernels, the whole network's forward and backward passes, and
Adam) with the FP64 oracle (oracle/unet.py), through the C ABI.

Both sides see the same BF16-rounded inputs and weights.  The GPU
accumulates in FP32 and rounds stored activations to BF16; the oracle
accumulates in FP64 and rounds at the same points.  Tolerances: a single
convolution's BF16 output within relative L2 1e-2 (one BF16 rounding is
2^-9 relative, and a few values on either side of a rounding boundary
differ by one BF16 step); FP32 weight gradients of one layer within 1e-3
(accumulation order only); the network's output and its parameter gradient
within 1e-2 (BF16 rounding differences carried through 17 layers); Adam
within 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import unet as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def un():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import unet
    return unet


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def bf(x):
    """Host float64 array already on the BF16 grid -> CUDA bfloat16."""
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).cuda()


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


CONV_CASES = [  # B, H, W, cin, cout
    (1, 128, 128, 32, 32),
    (2, 64, 64, 32, 64),
    (2, 32, 32, 64, 128),
    (4, 16, 16, 128, 256),
    (1, 32, 32, 256, 128),
    (2, 16, 64, 64, 32),
    # more tiles than resident CTAs: each persistent CTA takes several tiles
    # through both tensor-memory accumulators
    (8, 256, 256, 32, 32),
    (4, 128, 128, 64, 128),
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_forward_matches_oracle(un, case):
    B, H, W, ci, co = case
    rng = np.random.default_rng(sum(case))
    x = U.bf16(rng.standard_normal((B, H, W, ci)))
    Wt = U.bf16(rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci)))
    b = U.fp32(rng.standard_normal(co) * 0.1)
    out = un.conv3x3(bf(x), bf(Wt.reshape(co, 9, ci)),
                     torch.tensor(b, dtype=torch.float32).cuda(), op=un.OP_RELU)
    ref = U.bf16(np.maximum(U.conv3x3(x, Wt, b), 0.0))
    assert rel(host(out), ref) <= 1e-2, rel(host(out), ref)
    # most values are exactly the oracle's BF16 value
    assert np.mean(host(out) == ref) > 0.9


@pytest.mark.parametrize("case", CONV_CASES[:4])
def test_conv_data_gradient_with_mask_matches_oracle(un, case):
    """The data gradient: the same kernel on dy with the mirrored transposed
    weights w'[ci][8 - tap][co] = w[co][tap][ci], masked by the ReLU of the
    layer's input."""
    B, H, W, ci, co = case
    rng = np.random.default_rng(7 + sum(case))
    x = U.bf16(np.maximum(rng.standard_normal((B, H, W, ci)), 0.0))  # a ReLU output
    Wt = U.bf16(rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci)))
    dy = U.bf16(rng.standard_normal((B, H, W, co)))
    dx, _, _ = U.conv3x3_backward(x, Wt, dy)
    ref = U.bf16(dx * (x > 0))
    wt = Wt.reshape(co, 9, ci)[:, ::-1, :].transpose(2, 1, 0)  # [ci][tap'][co]
    got = un.conv3x3(bf(dy), bf(np.ascontiguousarray(wt)), None, op=un.OP_MASK, mask=bf(x))
    assert rel(host(got), ref) <= 1e-2, rel(host(got), ref)


WGRAD_CASES = [  # B, H, W, cin, cout
    (1, 128, 128, 32, 32),    # 64-byte swizzle for both operands, 3 row tiles
    (2, 64, 64, 32, 64),
    (2, 32, 32, 64, 128),     # 5 row tiles (the last half used)
    (4, 16, 16, 256, 256),    # 18 row tiles, 16-pixel rows
    (2, 64, 32, 128, 64),
]


@pytest.mark.parametrize("case", WGRAD_CASES)
def test_wgrad_matches_oracle(un, case):
    B, H, W, ci, co = case
    rng = np.random.default_rng(11 + sum(case))
    x = U.bf16(rng.standard_normal((B, H, W, ci)))
    dy = U.bf16(rng.standard_normal((B, H, W, co)))
    _, dW, _ = U.conv3x3_backward(x, np.zeros((co, 3, 3, ci)), dy)
    got = un.conv3x3_wgrad(bf(x), bf(dy))
    ref = dW.reshape(co, 9, ci)
    assert rel(got.cpu().numpy(), ref) <= 1e-3, rel(got.cpu().numpy(), ref)


def net_inputs(seed, B=2, H=128, W=128, in_ch=2):
    rng = np.random.default_rng(seed)
    theta = U.init_params(seed)
    inp = rng.standard_normal((B, H, W, in_ch)) * 0.5
    target = rng.standard_normal((B, H, W)) * 0.1
    return U.fp32(theta), U.fp32(inp), U.fp32(target)


def test_network_forward_matches_oracle(un):
    theta, inp, _ = net_inputs(3)
    B, H, W, c = inp.shape
    s = un.shape(B, H, W, c)
    out = un.forward(s, torch.tensor(theta, dtype=torch.float32).cuda(),
                     torch.tensor(inp, dtype=torch.float32).cuda())
    ref, _ = U.forward(theta, inp, rounding=True)
    assert rel(out.cpu().numpy(), ref) <= 1e-2, rel(out.cpu().numpy(), ref)


def test_network_gradient_matches_oracle(un):
    theta, inp, target = net_inputs(4)
    B, H, W, c = inp.shape
    s = un.shape(B, H, W, c)
    loss, grad, out = un.gradient(s, torch.tensor(theta, dtype=torch.float32).cuda(),
                                  torch.tensor(inp, dtype=torch.float32).cuda(),
                                  torch.tensor(target, dtype=torch.float32).cuda())
    Lref, gref, oref = U.loss_and_grad(theta, inp, target, rounding=True)
    assert rel(out.cpu().numpy(), oref) <= 1e-2
    assert abs(loss.item() - Lref) <= 1e-2 * Lref
    g = grad.cpu().numpy().astype(np.float64)
    assert rel(g, gref) <= 1e-2, rel(g, gref)
    # every layer's weights and biases, not only the total
    P, Q = U.unpack(g), U.unpack(gref)
    for name, _, _ in U.LAYERS:
        assert rel(P[name][0], Q[name][0]) <= 3e-2, (name, rel(P[name][0], Q[name][0]))
        assert rel(P[name][1], Q[name][1]) <= 3e-2, (name, rel(P[name][1], Q[name][1]))
    assert rel(P["head"][0], Q["head"][0]) <= 1e-2


def test_adam_matches_oracle(un):
    rng = np.random.default_rng(9)
    n = 100003
    th, g = U.fp32(rng.standard_normal(n)), U.fp32(rng.standard_normal(n))
    m, v = U.fp32(rng.standard_normal(n) * 0.1), U.fp32(rng.random(n) * 0.1)
    T = [torch.tensor(a, dtype=torch.float32).cuda() for a in (th, g, m, v)]
    un.adam(T[0], T[1], T[2], T[3], step=3, lr=1e-3)
    rth, rm, rv = U.adam(th, g, m, v, 3, lr=1e-3)
    assert rel(T[0].cpu().numpy(), rth) <= 1e-6
    assert rel(T[2].cpu().numpy(), rm) <= 1e-6 and rel(T[3].cpu().numpy(), rv) <= 1e-6


def test_training_steps_reduce_the_loss(un):
    """Adam on one fixed batch: the loss falls (the gradient points downhill
    through every layer)."""
    theta, inp, target = net_inputs(5)
    B, H, W, c = inp.shape
    s = un.shape(B, H, W, c)
    th = torch.tensor(theta, dtype=torch.float32).cuda()
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    x = torch.tensor(inp, dtype=torch.float32).cuda()
    t = torch.tensor(target, dtype=torch.float32).cuda()
    ws = un.alloc_workspace(s, True)
    losses = []
    for step in range(1, 31):
        loss, grad, _ = un.gradient(s, th, x, t, ws=ws)
        losses.append(loss.item())
        un.adam(th, grad, m, v, step, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0], losses
