"""``torch.autograd.Function`` over the C ABI: acoustic modelling whose
backward pass is the library's exact discrete adjoint.

``AcousticModelling.apply(v, wavelet, problem, src, rec)`` returns the
seismograms ``[nshot][1][nrec][nt]``; any scalar loss of them can be
differentiated with respect to the interior velocity ``v`` (through
``sweep_gradient`` with the data-space gradient passed as the residual) and
the wavelets (through ``sweep_adjoint``, the data are linear in them).  This
is the differentiable-solver use of Sec. 1 of the paper with the adjoint
written by hand instead of taped.

The velocity gradient is taken with the absorbing-border padding and the
CPML profile held fixed (the library's definition): it is exact for
perturbations of interior cells that do not move the edge-replicated border.
A padded model (``F_PADDED_MODEL``) can be modelled and differentiated with
respect to the wavelets, but not with respect to ``v``: its border cells are
inputs of their own, and the library gives no gradient for them.
"""
from __future__ import annotations

import copy

import torch

from . import sweep


def _check_differentiable(problem) -> None:
    if int(problem.flags) & sweep.F_PADDED_MODEL:
        raise ValueError("acoustic_modelling: no velocity gradient for a padded model "
                         "(F_PADDED_MODEL); pass the interior model to differentiate "
                         "with respect to v")


class AcousticModelling(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, wavelet, problem, src, rec):
        data = sweep.sweep_forward(problem, v.contiguous(), wavelet.contiguous(), src, rec)
        ctx.problem = problem
        ctx.save_for_backward(v, wavelet, src, rec)
        return data

    @staticmethod
    def backward(ctx, grad_data):
        v, wavelet, src, rec = ctx.saved_tensors
        g = grad_data.contiguous()
        grad_v = grad_w = None
        if ctx.needs_input_grad[0]:
            _check_differentiable(ctx.problem)
            p = copy.copy(ctx.problem)
            p.flags = int(p.flags) | sweep.F_RESIDUAL_IN
            grad_v, _, _ = sweep.sweep_gradient(p, v.contiguous(), wavelet.contiguous(), src, rec,
                                                g)
        if ctx.needs_input_grad[1]:
            grad_w = sweep.sweep_adjoint(ctx.problem, v.contiguous(), g, src, rec)
        return grad_v, grad_w, None, None, None


def acoustic_modelling(v, wavelet, problem, src, rec):
    """Differentiable acoustic forward modelling (see AcousticModelling)."""
    if v.requires_grad:
        _check_differentiable(problem)
    return AcousticModelling.apply(v, wavelet, problem, src, rec)
