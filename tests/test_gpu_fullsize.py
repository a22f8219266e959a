"""The benchmark's workload at full size: 301 x 901 interior + 40-cell CPML
(381 x 981 padded), dx 10 m, dt 1 ms, nt 3000, 20 shots, 301 receivers,
10 Hz, in the launch configuration the benchmark times (one sweep_gradient
call over all 20 shots).

* seismograms of the two edge shots (sources at x = 0 and x = 900, next to
  the absorbing border) against the FP64 oracle, which computes them in
  ~40 s on the host (relative L2 <= 1e-4, the parity bar of the
  seismograms);
* the 20-shot gradient against central finite differences of the GPU
  misfit along two smooth perturbations and along the gradient itself
  (relative 1e-2, as in the small cases): a property that holds at any
  size.  The gradient is d J / d v on interior cells with the border values
  and the CPML reference velocity held fixed, so the differences use a
  padded model (SWEEP_F_PADDED_MODEL) perturbed on the interior only and a
  fixed v_pml; the kernels and their launch shapes are those of the
  benchmark's call;
* the dot-product test of the forward map F: w -> d and sweep_adjoint at
  full size, <F w, F w> = <w, F^T (F w)> (relative 1e-5: FP32 wavefields,
  FP64 reductions).  With d = F w the sum does not cancel: against white
  noise d the 18 million terms of <F w, d> cancel to a value whose FP32
  rounding reaches ~2e-5 of it, which says nothing about the adjoint.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_14189_gb300 import inputs
from parity_util import worst_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import sweep
    w = inputs.workload_marmousi(nshot=20, nt=3000)
    nshot, nt, nrec = 20, 3000, w["rec"].shape[1]
    p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                      nshot=nshot, nrec=nrec, f_ref=w["f0"])
    dev = "cuda"
    wav = np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot).astype(np.float32)
    t = dict(v0=torch.tensor(w["model"], dtype=torch.float32, device=dev),
             vt=torch.tensor(w["v_true"], dtype=torch.float32, device=dev),
             wav=torch.tensor(wav, device=dev), src=torch.tensor(w["src"], device=dev),
             rec=torch.tensor(w["rec"], device=dev))
    return sweep, p, w, wav, t


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_edge_shot_seismograms_match_oracle(env):
    sweep, p, w, wav, t = env
    d = sweep.sweep_forward(p, t["v0"], t["wav"], t["src"], t["rec"]).cpu().numpy()[:, 0]
    pick = [0, 19]
    assert list(w["src"][pick, 1]) == [0, 900]
    q = oracle.make_problem(0, w["nz"], w["nx"], w["pml"], np.float32(w["dx"]),
                            np.float32(w["dt"]), p.nt, len(pick), p.nrec, np.float32(w["f0"]))
    oracle.set_threads(len(pick))
    ref = oracle.acoustic_forward(q, np.float32(w["model"]).astype(np.float64),
                                  wav[pick].astype(np.float64), w["src"][pick], w["rec"][pick])
    for j, s in enumerate(pick):
        assert rel(d[s], ref[j]) <= 1e-4, (s, rel(d[s], ref[j]))
        assert worst_trace(d[s], ref[j]) <= 1e-3, (s, worst_trace(d[s], ref[j]))


def test_full_gradient_finite_differences(env):
    sweep, p0, w, wav, t = env
    P, nz, nx = w["pml"], w["nz"], w["nx"]
    p = sweep.problem(nz=nz, nx=nx, pml=P, dx=w["dx"], dt=w["dt"], nt=p0.nt, nshot=p0.nshot,
                      nrec=p0.nrec, f_ref=w["f0"], v_pml=4600.0, flags=sweep.F_PADDED_MODEL)

    def padded(v):
        return torch.tensor(inputs.pad_edge(np.asarray(v, dtype=np.float64), P),
                            dtype=torch.float32, device="cuda")

    v0 = padded(w["model"])
    d_obs = sweep.sweep_forward(p, padded(w["v_true"]), t["wav"], t["src"], t["rec"])
    ws = sweep.alloc_workspace(p, sweep.MODE_GRADIENT)
    g, J, _ = sweep.sweep_gradient(p, v0, t["wav"], t["src"], t["rec"], d_obs, ws=ws)
    g = g.double().cpu().numpy()
    assert g.shape == (nz, nx) and np.isfinite(J.item()) and J.item() > 0
    pert = list(inputs.smooth_perturbations(nz, nx, w["model"], 2, seed=12))
    pert.append(0.01 * w["model"] * g / np.abs(g).max())  # along the gradient
    for k, pk in enumerate(pert):
        dv = np.zeros((nz + 2 * P, nx + 2 * P))
        dv[P:P + nz, P:P + nx] = pk
        dv = torch.tensor(dv, dtype=torch.float32, device="cuda")
        h = 0.5  # the perturbation is 1 % of v; step 0.5 of it
        Js = []
        for sgn in (1, -1):
            _, Jk, _ = sweep.sweep_gradient(p, v0 + sgn * h * dv, t["wav"], t["src"], t["rec"],
                                            d_obs, ws=ws)
            Js.append(Jk.item())
        fd = (Js[0] - Js[1]) / (2 * h)
        an = float(np.sum(g * pk))
        assert abs(fd - an) <= 1e-2 * abs(an), (k, fd, an)


def test_full_size_dot_product(env):
    sweep, p, w, wav, t = env
    rng = np.random.default_rng(21)
    wr = torch.tensor(rng.standard_normal((p.nshot, p.nt)), dtype=torch.float32,
                      device="cuda")
    Fw = sweep.sweep_forward(p, t["v0"], wr, t["src"], t["rec"])
    dr = Fw.clone()
    Ftd = sweep.sweep_adjoint(p, t["v0"], dr, t["src"], t["rec"])
    lhs = sweep.sweep_dot(Fw.reshape(-1), dr.reshape(-1)).item()
    rhs = sweep.sweep_dot(wr.reshape(-1), Ftd.reshape(-1)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
