"""Host logic of the learned preconditioner's FWI loop (CPU): the learned
direction is tried only when it agrees with the plain preconditioned
direction, kept only when the misfit confirms it, and the plain direction
is the fallback; the loop stops at the target model error; the training
pairs' normalisations; the initial weights' layout."""
import numpy as np
import pytest
import torch

from paper_2604_14189_gb300 import fwi


class _Quadratic:
    """Stand-in for the solver: J = 1/2 |m - m*|^2, non-uniform illumination."""

    def __init__(self):
        g = torch.Generator().manual_seed(3)
        self.target = 2000.0 + 300.0 * torch.rand(8, 8, generator=g)
        self.illum = 0.5 + torch.rand(8, 8, generator=g)
        self.calls = []  # want_illum of every gradient request

    def misfit(self, m):
        return 0.5 * float(((m.double() - self.target.double()) ** 2).sum())

    def gradient(self, m, want_illum=True):
        self.calls.append(want_illum)
        return (m - self.target), self.misfit(m), self.illum.clone() if want_illum else None


def _fake_fwi(q):
    f = object.__new__(fwi.Fwi)
    f.gradient, f.misfit = q.gradient, q.misfit
    return f


class _Pre:
    """Stand-in network: returns a fixed transform of the gradient."""

    def __init__(self, fn):
        self.fn = fn

    def direction(self, g, v):
        d = self.fn(g)
        return d / d.abs().max()


@pytest.fixture(scope="module")
def precond():
    pytest.importorskip("torch")
    from paper_2604_14189_gb300 import precond as p  # loads the library (no launch)
    return p


def _cfg():
    return fwi.FwiConfig(iterations=6, step=40.0, vmin=1000.0, vmax=4000.0)


def test_good_learned_direction_is_used(precond):
    q = _Quadratic()
    m0 = torch.full((8, 8), 2150.0)
    # the exact descent direction -(m - m*): agrees with the plain one, improves the misfit
    model, hist = precond.run_learned(_fake_fwi(q), _Pre(lambda g: -g), m0, _cfg(), q.target)
    assert all(h["used"] == "learned" for h in hist)
    assert hist[-1]["misfit_after"] < hist[0]["misfit"]
    assert all(h["cosine"] > 0.5 for h in hist)


def test_disagreeing_direction_falls_back_to_plain(precond):
    q = _Quadratic()
    m0 = torch.full((8, 8), 2150.0)
    # the ascent direction: its cosine with the plain direction is negative
    model, hist = precond.run_learned(_fake_fwi(q), _Pre(lambda g: g), m0, _cfg(), q.target,
                                      cos_min=0.0)
    assert all(h["used"] == "plain" for h in hist)
    assert all(h["cosine"] < 0 for h in hist)
    assert hist[-1]["misfit_after"] < hist[0]["misfit"]


def test_unconfirmed_learned_step_falls_back_to_plain(precond):
    """A direction that passes the cosine gate (cos_min = -1) but raises the
    misfit at every trial step is rejected by the line search; the plain
    direction then takes the iteration, and its trials count too."""
    q = _Quadratic()
    m0 = torch.full((8, 8), 2150.0)
    model, hist = precond.run_learned(_fake_fwi(q), _Pre(lambda g: g), m0, _cfg(), q.target,
                                      cos_min=-1.0)
    assert all(h["used"] == "plain" for h in hist)
    cfg = _cfg()
    assert all(h["trials"] > cfg.max_halvings + 1 for h in hist)


def test_stops_at_target_error(precond):
    q = _Quadratic()
    m0 = torch.full((8, 8), 2150.0)
    e0 = precond.model_error(m0, q.target)
    _, hist = precond.run_learned(_fake_fwi(q), _Pre(lambda g: -g), m0, _cfg(), q.target,
                                  target_error=0.9 * e0)
    assert hist[-1]["model_error"] <= 0.9 * e0
    assert len(hist) < _cfg().iterations
    assert precond.seconds_to(hist, 0.9 * e0) == hist[-1]["seconds"]
    assert precond.seconds_to(hist, -1.0) is None


def test_pair_normalisations(precond):
    g = torch.tensor([[2.0, -4.0], [1.0, 0.0]])
    v = torch.tensor([[1500.0, 3000.0], [4500.0, 3000.0]])
    x = precond.make_input(g, v)
    assert x.shape == (2, 2, 2)
    assert torch.allclose(x[..., 0], g / 4.0)
    assert torch.allclose(x[..., 1], torch.tensor([[-1.0, 0.0], [1.0, 0.0]]))
    illum = torch.tensor([[1.0, 3.0], [0.0, 9.0]])
    y = precond.make_target(g, illum, eps=0.1)
    raw = g / (illum + 0.9)
    assert torch.allclose(y, raw / raw.abs().max())
    # the target is the negative of the plain FWI direction
    assert torch.allclose(y, -fwi.precondition(g, illum, 0.1))


def test_init_params_layout(precond):
    """The product's initial weights: one flat vector in the library's layout,
    He-scaled weights and zero biases (every layer's first bias is zero, the
    weights around it are not)."""
    from paper_2604_14189_gb300 import unet
    th = precond.init_params(0, device="cpu")
    assert th.numel() == unet.PARAMS
    layers = [(32, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256),
              (256, 256), (256, 128), (256, 128), (128, 128), (128, 64), (128, 64), (64, 64),
              (64, 32), (64, 32), (32, 32)]
    k = 0
    for ci, co in layers:
        w = th[k:k + co * 9 * ci]
        assert abs(float(w.std()) - np.sqrt(2.0 / (9 * ci))) < 0.1 * np.sqrt(2.0 / (9 * ci))
        k += co * 9 * ci
        assert float(th[k:k + co].abs().max()) == 0.0
        k += co
    assert k + 33 == unet.PARAMS


def test_learned_iterations_skip_the_illumination(precond):
    """A trusted network needs the illumination only on judging iterations
    (the first and every judge_every-th); an untrusted one gets it with every
    gradient (the plain fallback), and a learned step the misfit rejects
    asks for it once more."""
    q = _Quadratic()
    m0 = torch.full((8, 8), 2150.0)
    cfg = fwi.FwiConfig(iterations=7, step=40.0, vmin=1000.0, vmax=4000.0)
    _, hist = precond.run_learned(_fake_fwi(q), _Pre(lambda g: -g), m0, cfg, q.target,
                                  judge_every=3)
    assert q.calls == [True, False, False, True, False, False, True]
    assert [h["judged"] for h in hist] == q.calls
    q2 = _Quadratic()
    _, hist = precond.run_learned(_fake_fwi(q2), _Pre(lambda g: g), m0, cfg, q2.target,
                                  judge_every=3)
    # distrusted from the first check on: every gradient comes with it
    assert q2.calls == [True] * 7
    assert all(h["used"] == "plain" for h in hist)
    q3 = _Quadratic()
    _, hist = precond.run_learned(_fake_fwi(q3), _Pre(lambda g: g), m0, cfg, q3.target,
                                  judge_every=3, cos_min=-1.0)
    # trusted but rejected by the misfit: the fallback asks for it again
    assert q3.calls == [True, False, True, False, True, True, False, True, False, True, True]
    assert all(h["used"] == "plain" for h in hist)
