"""The learned preconditioner end to end on the GPU, on a small case: pairs
from the solver are the (input, target) normalisations of the solver's own
gradient and illumination; a few epochs of training lower the loss; the
trained network plugs into the FWI loop, which lowers the misfit."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import fwi, inputs, precond, sweep
    return fwi, inputs, precond, sweep


def test_pairs_training_and_learned_fwi(env):
    fwi, inputs, precond, sweep = env
    n, nshot, nt = 128, 4, 500
    ps = precond.generate_pairs(10, seed=77, n=n, nshot=nshot, nt=nt)
    assert ps.inputs.shape == (10, n, n, 2) and ps.targets.shape == (10, n, n)
    # the pair is the solver's gradient and illumination, normalised
    p, wav, src, rec = precond.solver_setup(n, nshot, nt, "cuda")
    vt, vs = next(iter(inputs.precond_models(1, 77, n)))
    vt = torch.tensor(vt, dtype=torch.float32, device="cuda")
    vs = torch.tensor(vs, dtype=torch.float32, device="cuda")
    d = sweep.sweep_forward(p, vt, wav, src, rec)
    g, _, il = sweep.sweep_gradient(p, vs, wav, src, rec, d, want_illum=True)
    assert torch.allclose(ps.inputs[0], precond.make_input(g, vs), atol=1e-5)
    assert torch.allclose(ps.targets[0], precond.make_target(g, il), atol=1e-5)
    assert float(ps.targets.abs().amax(dim=(1, 2)).min()) == pytest.approx(1.0)
    # training lowers the loss
    tr = precond.train(ps.inputs, ps.targets, epochs=6, batch=3, lr=2e-3, seed=0, val_frac=0.1)
    losses = [e["train_loss"] for e in tr.epochs]
    assert losses[-1] < losses[0], losses
    # the learned loop runs through the solver and lowers the misfit
    pre = precond.Preconditioner(tr.theta, n)
    dl = pre.direction(g, vs)
    assert float(dl.abs().max()) == pytest.approx(1.0)
    inv = fwi.Fwi(p, wav, src, rec, d)
    cfg = fwi.FwiConfig(iterations=3, step=50.0, vmin=1400.0, vmax=4700.0)
    _, hist = precond.run_learned(inv, pre, vs, cfg, vt)
    inv.close()
    assert hist[-1]["misfit_after"] < hist[0]["misfit"]
    assert all(h["used"] in ("learned", "plain") for h in hist)
    assert all(np.isfinite(h["cosine"]) for h in hist)
