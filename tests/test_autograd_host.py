"""Host-side checks of the autograd wrapper (CPU, no launch): a padded
model has no velocity gradient, so asking for one is an error before any
work is done."""
import pytest
import torch

from paper_2604_14189_gb300 import autograd, sweep


def test_padded_model_velocity_gradient_rejected():
    p = sweep.problem(nz=8, nx=9, pml=2, dx=10.0, dt=1e-3, nt=5, nshot=1, nrec=1,
                      flags=sweep.F_PADDED_MODEL)
    v = torch.full((12, 13), 2000.0, requires_grad=True)
    w = torch.zeros(1, 5)
    src = torch.zeros(1, 2, dtype=torch.int32)
    rec = torch.zeros(1, 1, 2, dtype=torch.int32)
    with pytest.raises(ValueError, match="padded model"):
        autograd.acoustic_modelling(v, w, p, src, rec)
