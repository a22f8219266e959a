"""Full-waveform inversion loop over the C ABI.

FWI is the inversion use of the solver (Sec. 1; the FWI examples of Sec. 3):
update the velocity model along the negative misfit gradient until the
modelled data fit the observed data.  This module runs that loop with

* the gradient and the illumination I = sum over shots and steps of u^2
  from one ``sweep_gradient`` call (the illumination is accumulated inside
  the backward stencil kernel);
* the illumination-preconditioned direction d = -g / (I + eps max I),
  scaled so that max |d| = 1 (a step is then a velocity change in m/s);
* a backtracking line search with misfit confirmation: a trial model is
  accepted only if the solver's misfit of that model is lower than the
  current one; otherwise the step is halved (at most ``max_halvings`` times)
  and the model is kept if no trial improves;
* a bound constraint vmin <= v <= vmax on every trial.

The misfit of a trial model is J = 1/2 |d - d_obs|^2 from ``sweep_forward``
and three FP64 dot products of the library (no host round trip of the data).
The line search and the preconditioner are host logic, testable without a
GPU (``line_search`` takes any misfit function).

With ``checkpoint=<directory>``, ``run`` writes the state after every
iteration (``model.npy``: the current model; ``state.json``: the iterations
done, the next first-trial step and the history) and, called again with the
same directory, resumes from it: the iterations already done are not
repeated, and the step carries on from where it stopped.  Each file is
written to a temporary name and renamed into place, so an interrupted
write leaves the previous state whole.

With ``graphs=True`` (the default) the gradient call and the trial-misfit
calls (forward + two dot products) are recorded once as CUDA graphs over
fixed buffers; each evaluation copies the model into its buffer and replays
the graph, so an iteration costs a few host calls instead of tens of
thousands of launches.
"""
from __future__ import annotations

import dataclasses
import json
import os
import time
from typing import Callable

import numpy as np
import torch

from . import sweep


@dataclasses.dataclass
class FwiConfig:
    iterations: int = 20
    step: float = 50.0       # first trial: largest velocity change, m/s
    eps: float = 1e-2        # illumination stabiliser, relative to max I
    vmin: float = 1000.0
    vmax: float = 6000.0
    max_halvings: int = 5
    grow: float = 1.5        # step growth after a first-trial acceptance


def precondition(grad: torch.Tensor, illum: torch.Tensor, eps: float) -> torch.Tensor:
    """Descent direction -g / (I + eps max I), scaled to max |d| = 1."""
    d = -grad / (illum + eps * illum.max())
    m = d.abs().max()
    return d / m if float(m) > 0 else d


def line_search(misfit: Callable[[torch.Tensor], float], model: torch.Tensor,
                direction: torch.Tensor, j0: float, step: float, max_halvings: int,
                vmin: float, vmax: float):
    """Backtracking with misfit confirmation.  Returns (model, misfit, step
    of the accepted trial (or the last tried), trials, accepted)."""
    for k in range(max_halvings + 1):
        trial = (model + step * direction).clamp_(vmin, vmax)
        j = misfit(trial)
        if j < j0:
            return trial, j, step, k + 1, True
        step *= 0.5
    return model, j0, step, max_halvings + 1, False


STATE_VERSION = 1


def save_state(directory: str, model: torch.Tensor, done: int, step: float,
               history: list) -> None:
    """Writes the loop state after `done` iterations (model as float32
    ``.npy``, the rest as JSON); the model file is replaced first and the
    JSON last, so the JSON never names a model that is not on disk."""
    os.makedirs(directory, exist_ok=True)
    mpath = os.path.join(directory, "model.npy")
    tmp = mpath + ".tmp.npy"
    np.save(tmp, model.detach().to("cpu", torch.float32).numpy())
    os.replace(tmp, mpath)
    spath = os.path.join(directory, "state.json")
    with open(spath + ".tmp", "w") as f:
        json.dump({"version": STATE_VERSION, "iterations_done": int(done), "step": float(step),
                   "shape": list(model.shape), "history": history}, f)
    os.replace(spath + ".tmp", spath)


def load_state(directory: str):
    """(model as a CPU float32 tensor, iterations done, step, history), or
    None if the directory holds no state."""
    spath = os.path.join(directory, "state.json")
    if not os.path.exists(spath):
        return None
    with open(spath) as f:
        st = json.load(f)
    if st.get("version") != STATE_VERSION:
        raise ValueError(f"fwi state in {directory}: unknown version {st.get('version')}")
    model = torch.from_numpy(np.load(os.path.join(directory, "model.npy")))
    if list(model.shape) != st["shape"]:
        raise ValueError(f"fwi state in {directory}: model shape {list(model.shape)} "
                         f"does not match {st['shape']}")
    return model, int(st["iterations_done"]), float(st["step"]), list(st["history"])


class Fwi:
    """FWI of one acoustic problem: fixed geometry, wavelets and observed data."""

    def __init__(self, problem: sweep.Problem, wavelet, src, rec, d_obs, graphs: bool = True):
        self.p = problem
        self.wavelet, self.src, self.rec, self.d_obs = wavelet, src, rec, d_obs
        dev = d_obs.device
        self.ws_g = sweep.alloc_workspace(problem, sweep.MODE_GRADIENT, dev)
        self.ws_f = sweep.alloc_workspace(problem, sweep.MODE_FORWARD, dev)
        self.data = torch.empty_like(d_obs)
        self.dd_obs = float(sweep.sweep_dot(d_obs.reshape(-1), d_obs.reshape(-1)))
        self._gg = self._gg0 = self._gf = None
        if graphs:
            self._record(dev)

    def _record(self, dev):
        """Records the gradient call and the trial-misfit calls over fixed
        buffers (model in, results out)."""
        p = self.p
        shape = (p.nz, p.nx)
        self._mg = torch.empty(shape, dtype=torch.float32, device=dev)  # gradient model
        self._mt = torch.empty(shape, dtype=torch.float32, device=dev)  # trial model
        self._g = torch.empty(shape, dtype=torch.float32, device=dev)
        self._il = torch.empty(shape, dtype=torch.float32, device=dev)
        self._j = torch.empty((), dtype=torch.float64, device=dev)
        self._dd = torch.empty((), dtype=torch.float64, device=dev)
        self._do = torch.empty((), dtype=torch.float64, device=dev)
        d, do = self.data.reshape(-1), self.d_obs.reshape(-1)
        side = torch.cuda.Stream(dev)
        with sweep.capture(side) as c:
            sweep.sweep_gradient(p, self._mg, self.wavelet, self.src, self.rec, self.d_obs,
                                 grad=self._g, misfit=self._j, illum=self._il, ws=self.ws_g,
                                 stream=side)
        self._gg = c.graph
        with sweep.capture(side) as c:  # the same gradient without the illumination
            sweep.sweep_gradient(p, self._mg, self.wavelet, self.src, self.rec, self.d_obs,
                                 grad=self._g, misfit=self._j, ws=self.ws_g, stream=side)
        self._gg0 = c.graph
        with sweep.capture(side) as c:
            sweep.sweep_forward(p, self._mt, self.wavelet, self.src, self.rec, data=self.data,
                                ws=self.ws_f, stream=side)
            sweep.sweep_dot(d, d, out=self._dd, stream=side)
            sweep.sweep_dot(d, do, out=self._do, stream=side)
        self._gf = c.graph
        torch.cuda.current_stream(dev).wait_stream(side)

    def close(self) -> None:
        """Frees the recorded graphs (none of their replays may be pending)."""
        for g in (self._gg, self._gg0, self._gf):
            if g is not None:
                g.close()
        self._gg = self._gg0 = self._gf = None

    @staticmethod
    def _checked(ws):
        st = sweep.status(ws)
        if st != sweep.OK:
            raise sweep.SweepError(st, "fwi")

    def misfit(self, model: torch.Tensor) -> float:
        """J = 1/2 (<d, d> - 2 <d, d_obs> + <d_obs, d_obs>), FP64 sums."""
        if self._gf is not None:
            self._mt.copy_(model)
            self._gf.launch()
            self._checked(self.ws_f)
            return 0.5 * (float(self._dd) - 2.0 * float(self._do) + self.dd_obs)
        d = sweep.sweep_forward(self.p, model, self.wavelet, self.src, self.rec, data=self.data,
                                ws=self.ws_f)
        dd = float(sweep.sweep_dot(d.reshape(-1), d.reshape(-1)))
        do = float(sweep.sweep_dot(d.reshape(-1), self.d_obs.reshape(-1)))
        return 0.5 * (dd - 2.0 * do + self.dd_obs)

    def gradient(self, model: torch.Tensor, want_illum: bool = True):
        """(gradient, misfit, illumination or None) of `model`; new tensors.
        Without the illumination the backward pass skips its accumulation."""
        if self._gg is not None:
            self._mg.copy_(model)
            (self._gg if want_illum else self._gg0).launch()
            self._checked(self.ws_g)
            return (self._g.clone(), float(self._j),
                    self._il.clone() if want_illum else None)
        g, j, illum = sweep.sweep_gradient(self.p, model, self.wavelet, self.src, self.rec,
                                           self.d_obs, want_illum=want_illum, ws=self.ws_g)
        return g, float(j), illum

    def run(self, model0: torch.Tensor, cfg: FwiConfig,
            callback: Callable[[int, torch.Tensor, dict], None] | None = None,
            checkpoint: str | None = None):
        """Returns (model, history); history[i] = dict(misfit, step, trials,
        accepted, seconds) of iteration i (misfit before the update).  With
        `checkpoint`, resumes from the state saved there (if any) and saves
        the state after every iteration; `seconds` counts from the start of
        this call."""
        model = model0.clone().contiguous()
        step = cfg.step
        history = []
        start = 0
        if checkpoint is not None:
            saved = load_state(checkpoint)
            if saved is not None:
                m, start, step, history = saved
                if m.shape != model.shape:
                    raise ValueError("fwi: the saved model's shape differs from model0's")
                model = m.to(model0.device, model0.dtype).contiguous()
                if history and not history[-1]["accepted"]:
                    return model, history  # the saved run had already stopped
        t0 = time.perf_counter()
        for it in range(start, cfg.iterations):
            g, j, illum = self.gradient(model)
            d = precondition(g, illum, cfg.eps)
            model, jn, used, trials, ok = line_search(self.misfit, model, d, j, step,
                                                     cfg.max_halvings, cfg.vmin, cfg.vmax)
            model = model.contiguous()
            step = used * (cfg.grow if ok and trials == 1 else 1.0)
            rec = dict(misfit=j, misfit_after=jn, step=used, trials=trials, accepted=ok,
                       seconds=time.perf_counter() - t0)
            history.append(rec)
            if checkpoint is not None:
                save_state(checkpoint, model, it + 1, step, history)
            if callback is not None:
                callback(it, model, rec)
            if not ok:
                break
        return model, history
