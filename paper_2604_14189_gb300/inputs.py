"""Seeded synthetic inputs for the acoustic and elastic solvers.

This module holds no solver arithmetic: it only draws models, wavelets and
acquisition geometry (numpy + scipy on the host).  Both the CUDA path's tests
and the CPU oracle's tests take their inputs from here.

Workload recipes (the paper names no public dataset; every input is
synthetic):

* ``layered3`` -- 3 flat layers 1500/2500/3500 m/s with interfaces at
  z = 60 and 130 cells (acoustic single-shot forward, 200 x 200 interior).
* ``marmousi_like`` -- smooth layered gradient 1500 -> 4500 m/s with 8 seeded
  undulating interfaces (+-150 m/s) plus 5 Gaussian anomalies (+-10 %,
  sigma 15 cells); the starting model is the true one blurred with a 40-cell
  Gaussian (acoustic forward + adjoint gradient, 301 x 901 interior).
* ``elastic_layered`` -- Vp 1800 -> 5000 m/s linear in depth plus 10 seeded
  layers (+-200 m/s), Vs = Vp / 1.73, Gardner density 310 Vp^0.25.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import gaussian_filter


def ricker(f0: float, dt: float, nt: int, t0: float | None = None,
           shift: float = 0.0) -> np.ndarray:
    """Ricker wavelet sampled at t_n = (n + shift) dt, delay t0 = 1.5 / f0."""
    if t0 is None:
        t0 = 1.5 / f0
    t = (np.arange(nt) + shift) * dt - t0
    a = (np.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def surface_line(nshot: int, z: int, xs) -> np.ndarray:
    """[nshot][n][2] positions (z, x) with the same x list for every shot."""
    xs = np.asarray(xs, dtype=np.int32)
    pos = np.stack([np.full_like(xs, z), xs], axis=-1)
    return np.broadcast_to(pos, (nshot,) + pos.shape).copy()


def layered3(nz: int = 200, nx: int = 200) -> np.ndarray:
    v = np.empty((nz, nx), dtype=np.float64)
    z = np.arange(nz)[:, None]
    v[:] = np.where(z < 60, 1500.0, np.where(z < 130, 2500.0, 3500.0))
    return v


def marmousi_like(nz: int, nx: int, seed: int, vmin=1500.0, vmax=4500.0,
                  n_interfaces=8, n_anomalies=5, start_sigma=40.0):
    """True and starting velocity models (float64 [nz][nx]); the starting
    model is the true one blurred by a Gaussian of width start_sigma cells
    (None: no starting model is made)."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    v = vmin + (vmax - vmin) * z / max(nz - 1, 1) + 0.0 * x
    depths = np.sort(rng.uniform(0.1 * nz, 0.9 * nz, n_interfaces))
    for d in depths:
        jump = rng.choice([-150.0, 150.0])
        k = rng.uniform(1.0, 3.0) * 2 * np.pi / nx
        ph = rng.uniform(0, 2 * np.pi)
        surf = d + 5.0 * np.sin(k * x + ph)
        v = v + jump * (z >= surf)
    v = np.clip(v, vmin, vmax)
    for _ in range(n_anomalies):
        cz = rng.uniform(0.2, 0.8) * nz
        cx = rng.uniform(0.2, 0.8) * nx
        amp = rng.uniform(-0.1, 0.1)
        v = v * (1.0 + amp * np.exp(-((z - cz) ** 2 + (x - cx) ** 2) / (2 * 15.0 ** 2)))
    if start_sigma is None:
        return v, None
    return v, gaussian_filter(v, sigma=start_sigma, mode="nearest")


def smooth_perturbations(nz: int, nx: int, v: np.ndarray, count: int, seed: int,
                         sigma: float = 10.0, rel: float = 0.01) -> np.ndarray:
    """[count][nz][nx] blurred white noise scaled to `rel` of v (max norm)."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, nz, nx))
    for k in range(count):
        w = gaussian_filter(rng.standard_normal((nz, nx)), sigma=sigma, mode="nearest")
        out[k] = rel * v * w / np.abs(w).max()
    return out


def elastic_layered(nz: int, nx: int, seed: int, n_layers: int = 10):
    """(vp, vs, rho) float64 [3][nz][nx]."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz, dtype=np.float64)[:, None]
    vp = 1800.0 + (5000.0 - 1800.0) * z / max(nz - 1, 1) + np.zeros((1, nx))
    for d in np.sort(rng.uniform(0.05 * nz, 0.95 * nz, n_layers)):
        vp = vp + rng.uniform(-200.0, 200.0) * (z >= d)
    vp = np.clip(vp, 1800.0, 5000.0)
    vs = vp / 1.73
    rho = 310.0 * vp ** 0.25
    return np.stack([vp, vs, rho])


def pad_edge(model: np.ndarray, pml: int) -> np.ndarray:
    """Edge-replicate the last two axes by `pml` cells (model layout helper)."""
    pad = [(0, 0)] * (model.ndim - 2) + [(pml, pml), (pml, pml)]
    return np.pad(model, pad, mode="edge")


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def workload_layered3():
    """Acoustic forward, one shot: 200 x 200 + 40-cell CPML, nt = 1000."""
    nz = nx = 200
    return dict(nz=nz, nx=nx, pml=40, dx=10.0, dt=1e-3, nt=1000, f0=10.0,
                model=layered3(nz, nx),
                src=np.array([[2, 100]], dtype=np.int32),
                rec=surface_line(1, 2, np.arange(200)))


def surface_survey(nx: int, total_shots: int, rec_step: int = 3, z: int = 2):
    """A surface acquisition: `total_shots` sources at depth z evenly spaced
    over the whole width (x = round(linspace(0, nx - 1, total_shots))), and
    receivers at depth z every `rec_step` cells, the same for every shot."""
    sx = np.round(np.linspace(0, nx - 1, total_shots)).astype(np.int32)
    src = np.stack([np.full_like(sx, z), sx], axis=-1).astype(np.int32)
    return src, surface_line(total_shots, z, np.arange(0, nx, rec_step))


def workload_marmousi(nshot: int = 20, nt: int = 3000, seed: int = 1001,
                      total_shots: int = 20, shots: slice | None = None):
    """Acoustic forward + adjoint gradient: 301 x 901, nt = 3000.  The survey
    has `total_shots` surface shots (20: the single-GPU workload); `shots`
    selects a contiguous block of them (one rank's share), else the first
    `nshot`."""
    nz, nx = 301, 901
    v_true, v0 = marmousi_like(nz, nx, seed)
    src, rec = surface_survey(nx, total_shots)
    sl = shots if shots is not None else slice(0, nshot)
    return dict(nz=nz, nx=nx, pml=40, dx=10.0, dt=1e-3, nt=nt, f0=10.0,
                v_true=v_true, model=v0, src=src[sl], rec=rec[sl])


def workload_elastic(nshot: int = 64, nt: int = 4000, seed: int = 1002,
                     nz: int = 500, nx: int = 1500):
    """Elastic forward: 500 x 1500, dx = 5 m, dt = 0.5 ms, 64 shots, 750 receivers."""
    m = elastic_layered(nz, nx, seed)
    sx = np.round(np.linspace(0, nx - 1, 64)).astype(np.int32)[:nshot]
    src = np.stack([np.full_like(sx, 2), sx], axis=-1).astype(np.int32)
    rec = surface_line(nshot, 2, np.arange(0, nx, 2))
    return dict(nz=nz, nx=nx, pml=40, dx=5.0, dt=5e-4, nt=nt, f0=15.0,
                model=m, src=src, rec=rec)


def workload_fwi(seed: int = 1004, n: int = 256, nshot: int = 16, nt: int = 1500):
    """FWI on a seeded n x n layered + Gaussian-anomaly model (the generator
    of the 301 x 901 workload), dx = 10 m, nt = 1500, 16 surface shots,
    receivers at every surface cell, 10 Hz; starting model = the true model
    blurred with a 40-cell Gaussian."""
    v_true, v0 = marmousi_like(n, n, seed)
    sx = np.round(np.linspace(0, n - 1, nshot)).astype(np.int32)
    src = np.stack([np.full_like(sx, 2), sx], axis=-1).astype(np.int32)
    rec = surface_line(nshot, 2, np.arange(0, n))
    return dict(nz=n, nx=n, pml=40, dx=10.0, dt=1e-3, nt=nt, f0=10.0,
                v_true=v_true, model=v0, src=src, rec=rec)


def precond_models(count: int, seed: int, n: int = 256):
    """Models of the learned preconditioner's training pairs and of its
    held-out FWI tests: `count` seeded n x n layered + Gaussian-anomaly
    models (the FWI workload's generator, seeds seed, seed + 1, ...), each
    with a starting model blurred by a Gaussian of width U[10, 40] cells
    (so that gradients of early and later FWI iterations are represented).
    Yields (v_true, v_start)."""
    rng = np.random.default_rng(seed)
    for k in range(count):
        v_true, _ = marmousi_like(n, n, seed + k, start_sigma=None)
        sigma = float(rng.uniform(10.0, 40.0))
        yield v_true, gaussian_filter(v_true, sigma=sigma, mode="nearest")


def precond_heldout(count: int, seed: int = 900000, n: int = 256, sigma: float = 20.0):
    """Held-out FWI tests of the learned preconditioner: `count` seeded
    models of the same generator (seeds disjoint from the training pairs'),
    each with its starting model blurred by a `sigma`-cell Gaussian.  From
    20 cells plain FWI lowers the model error steadily over 20 iterations
    (from 40 cells, 20 iterations of 10 Hz surface data often raise it, so a
    comparison of time to a model error would be empty).  Yields
    (v_true, v_start)."""
    for k in range(count):
        yield marmousi_like(n, n, seed + k, start_sigma=sigma)


def workload_batch(seed: int = 1003, count: int = 256):
    """Heterogeneous batch: `count` seeded random layered models, interior
    nz, nx ~ U[128, 512], border 20..40 cells, nt ~ U[800, 3000], 1..8 shots,
    3..8 flat layers in [1500, 4500] m/s, dx = 10 m, dt = 1 ms, 10 Hz;
    sources at z = 2 evenly spaced, receivers at z = 2 in every cell."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nz, nx = int(rng.integers(128, 513)), int(rng.integers(128, 513))
        pml = int(rng.integers(20, 41))
        nt = int(rng.integers(800, 3001))
        ns = int(rng.integers(1, 9))
        nl = int(rng.integers(3, 9))
        tops = np.sort(rng.integers(1, nz, nl - 1))
        vel = np.sort(rng.uniform(1500.0, 4500.0, nl))
        z = np.arange(nz)[:, None] + np.zeros((1, nx))
        v = np.full((nz, nx), vel[0])
        for t, vv in zip(tops, vel[1:]):
            v[z >= t] = vv
        sx = np.round(np.linspace(0, nx - 1, ns)).astype(np.int32)
        src = np.stack([np.full_like(sx, 2), sx], axis=-1).astype(np.int32)
        rec = surface_line(ns, 2, np.arange(nx))
        out.append(dict(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, f0=10.0, model=v,
                        src=src, rec=rec))
    return out
