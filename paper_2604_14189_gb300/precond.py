"""Learned gradient preconditioner for FWI: the U-Net of ``unet.py`` trained
on pairs that the solver itself generates, and an FWI loop that uses it
only where the solver confirms it.

The paper integrates networks with its solvers (Sec. 1, Sec. 2.1) without
fixing one; this is the workload's choice of network and use.

Training pairs.  For a seeded layered + Gaussian-anomaly model (the
generator of the FWI workload) and a starting model blurred by a random
Gaussian width (so that gradients of early and later FWI iterations are
both represented), one ``sweep_gradient`` call gives the raw gradient g and
the illumination I = sum over shots and steps of u^2.  The pair is

    input  = [g / max|g|, (v - 3000) / 1500]      (2 channels, [H][W][2])
    target = p / max|p|,  p = g / (I + eps max I)  (the plain preconditioned
                                                    gradient)

Use in FWI (``run_learned``).  The network stands in for the illumination:
a learned iteration takes the gradient alone from the solver (the backward
pass then skips the illumination accumulation) and the direction
-net(input) / max|net(input)|.  The plain preconditioned gradient judges it
(every few iterations its cosine with the learned direction must be at
least ``cos_min`` for the network to stay trusted) and is the fallback: a
learned step that the solver's misfit does not confirm in the line search,
or an untrusted network, gives the iteration to the plain direction.

Everything that touches a tensor element runs in the library's kernels
(the solver, the U-Net's tcgen05 convolutions and Adam) or in torch's
element-wise GPU ops for the normalisations; this module is orchestration.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import fwi, inputs, sweep, unet

V_REF, V_SCALE = 3000.0, 1500.0


def init_params(seed: int, device=None) -> torch.Tensor:
    """He-normal initial weights (std sqrt(2 / fan_in)), zero biases, head
    weights with std sqrt(1 / 32); flat float32 vector on the GPU."""
    layers = [(32, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256),
              (256, 256), (256, 128), (256, 128), (128, 128), (128, 64), (128, 64), (64, 64),
              (64, 32), (64, 32), (32, 32)]
    g = torch.Generator().manual_seed(seed)
    parts = []
    for ci, co in layers:
        parts.append(torch.randn(co * 9 * ci, generator=g) * (2.0 / (9 * ci)) ** 0.5)
        parts.append(torch.zeros(co))
    parts.append(torch.randn(32, generator=g) * (1.0 / 32) ** 0.5)
    parts.append(torch.zeros(1))
    theta = torch.cat(parts).to(torch.float32)
    assert theta.numel() == unet.PARAMS
    return theta.to(device or "cuda")


def _unit(x: torch.Tensor) -> torch.Tensor:
    m = x.abs().max()
    return x / m if float(m) > 0 else x


def make_input(g: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """[H][W][2] network input of a gradient and its model."""
    return torch.stack([_unit(g), (v - V_REF) / V_SCALE], dim=-1).contiguous()


def make_target(g: torch.Tensor, illum: torch.Tensor, eps: float = 1e-2) -> torch.Tensor:
    """The plain preconditioned gradient g / (I + eps max I), max-normalised."""
    return _unit(g / (illum + eps * illum.max())).contiguous()


@dataclasses.dataclass
class PairSet:
    inputs: torch.Tensor    # [n][H][W][2]
    targets: torch.Tensor   # [n][H][W]
    seconds: float          # solver time spent generating them
    cell_steps: float       # padded cell-steps of fwd+adj solved (forward of d_obs excluded)


def solver_setup(n: int, nshot: int, nt: int, device):
    """Problem, wavelets and acquisition of the preconditioner's workload:
    n x n interior, 40-cell CPML, dx 10 m, dt 1 ms, 10 Hz Ricker, nshot
    surface shots, receivers at every surface cell."""
    w = inputs.workload_fwi(seed=0, n=n, nshot=nshot, nt=nt)
    p = sweep.problem(nz=n, nx=n, pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt, nshot=nshot,
                      nrec=w["rec"].shape[1], f_ref=w["f0"], v_pml=4500.0)
    wav = torch.tensor(np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot),
                       dtype=torch.float32, device=device)
    return p, wav, torch.tensor(w["src"], device=device), torch.tensor(w["rec"], device=device)


def generate_pairs(count: int, seed: int, n: int = 256, nshot: int = 16, nt: int = 1500,
                   device=None) -> PairSet:
    """`count` training pairs from the solver (see the module docstring)."""
    dev = torch.device(device or "cuda")
    p, wav, src, rec = solver_setup(n, nshot, nt, dev)
    ws_f = sweep.alloc_workspace(p, sweep.MODE_FORWARD, dev)
    ws_g = sweep.alloc_workspace(p, sweep.MODE_GRADIENT, dev)
    X = torch.empty((count, n, n, 2), dtype=torch.float32, device=dev)
    Y = torch.empty((count, n, n), dtype=torch.float32, device=dev)
    data = torch.empty((nshot, 1, p.nrec, nt), dtype=torch.float32, device=dev)
    grad = torch.empty((n, n), dtype=torch.float32, device=dev)
    illum = torch.empty((n, n), dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k, (vt, vs) in enumerate(inputs.precond_models(count, seed, n)):
        vt = torch.tensor(vt, dtype=torch.float32, device=dev)
        vs = torch.tensor(vs, dtype=torch.float32, device=dev)
        sweep.sweep_forward(p, vt, wav, src, rec, data=data, ws=ws_f)
        sweep.sweep_gradient(p, vs, wav, src, rec, data, grad=grad, illum=illum, ws=ws_g)
        X[k] = make_input(grad, vs)
        Y[k] = make_target(grad, illum)
    torch.cuda.synchronize(dev)
    NP = (n + 2 * p.pml) ** 2
    return PairSet(X, Y, time.perf_counter() - t0, float(count) * NP * nt * nshot)


@dataclasses.dataclass
class TrainResult:
    theta: torch.Tensor
    epochs: list            # per epoch: mean training loss, validation loss, seconds
    steps: int
    seconds: float


def evaluate(theta, X, Y, batch: int = 8) -> float:
    """Mean squared error of the network on (X, Y)."""
    n, H, W, c = X.shape
    tot = 0.0
    ws = None
    for i in range(0, n, batch):
        xb = X[i:i + batch].contiguous()
        s = unet.shape(xb.shape[0], H, W, c)
        if ws is None or ws.numel() < unet.workspace_bytes(s, False):
            ws = unet.alloc_workspace(s, False, X.device)
        out = unet.forward(s, theta, xb, ws=ws)
        tot += float(((out - Y[i:i + batch]) ** 2).sum())
    return tot / (n * H * W)


def train(X, Y, epochs: int = 20, batch: int = 8, lr: float = 1e-3, seed: int = 0,
          val_frac: float = 0.05, theta0=None) -> TrainResult:
    """Adam on the MSE loss over shuffled mini-batches; a fixed validation
    split is scored after every epoch.  Learning rate: cosine decay from lr
    to lr / 20."""
    n, H, W, c = X.shape
    nval = max(1, int(round(val_frac * n)))
    ntr = n - nval
    theta = init_params(seed, X.device) if theta0 is None else theta0.clone()
    m, v = torch.zeros_like(theta), torch.zeros_like(theta)
    s = unet.shape(batch, H, W, c)
    ws = unet.alloc_workspace(s, True, X.device)
    grad = torch.empty_like(theta)
    out = torch.empty((batch, H, W), dtype=torch.float32, device=X.device)
    loss = torch.empty((), dtype=torch.float64, device=X.device)
    rng = np.random.default_rng(seed)
    steps, hist = 0, []
    per_epoch = ntr // batch
    total = max(epochs * per_epoch, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for e in range(epochs):
        order = torch.tensor(rng.permutation(ntr), device=X.device)
        acc = torch.zeros((), dtype=torch.float64, device=X.device)
        for b in range(per_epoch):
            idx = order[b * batch:(b + 1) * batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            unet.gradient(s, theta, xb, yb, grad=grad, out=out, loss=loss, ws=ws, sync=False)
            acc += loss
            steps += 1
            lr_t = lr * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * steps / total)))
            unet.adam(theta, grad, m, v, steps, lr_t)
        st = sweep.status(ws)
        if st != sweep.OK:
            raise sweep.SweepError(st, "precond.train")
        hist.append(dict(epoch=e, train_loss=float(acc) / max(per_epoch, 1),
                         val_loss=evaluate(theta, X[ntr:], Y[ntr:]),
                         seconds=time.perf_counter() - t0))
    torch.cuda.synchronize()
    return TrainResult(theta, hist, steps, time.perf_counter() - t0)


class Preconditioner:
    """A trained network applied to one gradient at a time."""

    def __init__(self, theta: torch.Tensor, n: int, device=None):
        self.theta = theta
        self.s = unet.shape(1, n, n, 2)
        self.ws = unet.alloc_workspace(self.s, False, device or theta.device)
        self.out = torch.empty((1, n, n), dtype=torch.float32, device=theta.device)

    def direction(self, g: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
        """Learned descent direction, max |d| = 1."""
        x = make_input(g, v)[None]
        unet.forward(self.s, self.theta, x, out=self.out, ws=self.ws, sync=False)
        return _unit(-self.out[0])


def model_error(v: torch.Tensor, v_true: torch.Tensor) -> float:
    return float((v - v_true).norm() / v_true.norm())


def run_plain(inv: fwi.Fwi, model0, cfg: fwi.FwiConfig, v_true):
    """Plain illumination-preconditioned FWI; history with the model error
    and the wall time after every iteration."""
    hist = []

    def cb(it, model, rec):
        rec["model_error"] = model_error(model, v_true)
        hist.append(rec)

    model, _ = inv.run(model0, cfg, callback=cb)
    return model, hist


def run_learned(inv: fwi.Fwi, pre: Preconditioner, model0, cfg: fwi.FwiConfig, v_true,
                cos_min: float = 0.0, target_error: float | None = None, judge_every: int = 5):
    """FWI with the learned direction (module docstring); stops early once
    the model error reaches `target_error`.

    The network stands in for the illumination, so a learned iteration asks
    the solver for the gradient alone.  Every `judge_every`-th iteration
    (and the first) also computes the illumination and the plain direction,
    whose cosine with the learned one decides whether the learned direction
    is trusted until the next check (cos >= cos_min).  A learned step the
    solver's misfit does not confirm, or an untrusted network, falls back to
    the plain direction (with the illumination computed for it)."""
    model = model0.clone().contiguous()
    step, hist = cfg.step, []
    trusted, cos = True, float("nan")
    t0 = time.perf_counter()
    for it in range(cfg.iterations):
        judge = it % max(judge_every, 1) == 0
        need_plain = judge or not trusted
        g, j, illum = inv.gradient(model, want_illum=need_plain)
        d_plain = fwi.precondition(g, illum, cfg.eps) if need_plain else None
        if judge or trusted:
            d_learn = pre.direction(g, model)
        if judge:
            cos = float((d_learn * d_plain).sum() / (d_learn.norm() * d_plain.norm() + 1e-30))
            trusted = cos >= cos_min
        used, trials, ok = "plain", 0, False
        if trusted:
            m1, jn, st, k, ok = fwi.line_search(inv.misfit, model, d_learn, j, step,
                                                cfg.max_halvings, cfg.vmin, cfg.vmax)
            trials += k
            if ok:
                used = "learned"
        if used == "plain":
            if d_plain is None:
                g, j, illum = inv.gradient(model, want_illum=True)
                d_plain = fwi.precondition(g, illum, cfg.eps)
            m1, jn, st, k, ok = fwi.line_search(inv.misfit, model, d_plain, j, step,
                                                cfg.max_halvings, cfg.vmin, cfg.vmax)
            trials += k
        model = m1.contiguous()
        step = st * (cfg.grow if ok and k == 1 else 1.0)
        err = model_error(model, v_true)
        hist.append(dict(misfit=j, misfit_after=jn, step=st, trials=trials, accepted=ok,
                         used=used, judged=judge, cosine=cos, model_error=err,
                         seconds=time.perf_counter() - t0))
        if not ok or (target_error is not None and err <= target_error):
            break
    return model, hist


def seconds_to(hist, target: float):
    """Wall seconds at which the model error first reached `target` (None if
    it never did)."""
    for h in hist:
        if h["model_error"] <= target:
            return h["seconds"]
    return None
