"""Heterogeneous batches: many independent problems of uneven grid size,
border width, record length and shot count in one call (acoustic problems
share launches; elastic ones run one problem per call).

Batch modelling is the shot / model dimension of Sec. 2.2; the paper also
runs several velocity models at once.  Here every problem keeps its own
geometry and time loop, and the batch is made to fill the GPU by running
problems concurrently:

* each problem's stencil kernels are persistent with a grid of
  min(#SMs, work units), so a small problem occupies only some SMs and the
  others are free for concurrent problems;
* problems are dealt to ``streams`` CUDA streams, longest first, each to the
  stream with the least work queued so far (LPT list scheduling, within 4/3
  of the optimal makespan); the cost of a problem is its padded cell-steps
  (padded cells x nt x shots);
* every stream is fed by its own host thread: the C ABI releases the GIL,
  so the launches of the streams are issued in parallel and the host does
  not become the bottleneck of thousands of short time steps;
* a stream reuses one workspace (sized for its largest problem), and after
  every problem the library's status word is copied to a per-problem slot,
  so an error is attributed to its problem without synchronising.

With ``SWEEP_F_ONE_LAUNCH`` set on the items (all of them, for fused
runs) each cohort's forward and backward time loops run as one cooperative
launch each, and the cohorts run one after the other on one stream.

Gradients (``fused=True``, the default) go further: problems of similar
record length are grouped into cohorts of up to 16, and each cohort is one
``sweep_gradient_batch`` call whose every time-step launch carries the step
of all its problems (a problem past its record length drops out), so the
launches' fixed cost (about 6.5 us per half-step, larger than the work of a
small problem's step) is paid once per cohort, not once per problem.
Cohorts are dealt to the streams by the same LPT rule.

``autotune_streams`` times the batch (or a sample of it) for a few stream
counts and returns the fastest.  ``autotune_tiles`` then chooses the
stencil tile height per problem size: problems with fewer 32-row work
units than a threshold get 16-row tiles (``SWEEP_F_ROWS16``: twice the
units, so a small grid spreads over more SMs), and the threshold is timed
over a few candidates (0 = 32-row tiles everywhere).  Both keep their
results in the JSON file named by ``SWEEP_TUNE_CACHE``.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import os
import threading
import time

import torch

from . import sweep


@dataclasses.dataclass
class Item:
    """One problem: inputs on the GPU; outputs filled by ``run``."""
    problem: sweep.Problem
    model: torch.Tensor
    wavelet: torch.Tensor
    src: torch.Tensor
    rec: torch.Tensor
    d_obs: torch.Tensor | None = None   # gradient mode
    grad: torch.Tensor | None = None    # out (gradient mode)
    misfit: torch.Tensor | None = None  # out (gradient mode)
    data: torch.Tensor | None = None    # out (forward mode)


def out_shapes(p: sweep.Problem) -> tuple[tuple[int, ...], tuple[int, ...]]:
    """Shapes of (gradient, recorded data) of a problem: acoustic [nz][nx]
    and [nshot][1][nrec][nt]; elastic [3][nz][nx] (vp, vs, rho) and
    [nshot][2][nrec][nt] (vx, vz)."""
    if p.physics == sweep.ELASTIC:
        return (3, p.nz, p.nx), (p.nshot, 2, p.nrec, p.nt)
    return (p.nz, p.nx), (p.nshot, 1, p.nrec, p.nt)


def cost(p: sweep.Problem) -> int:
    """Padded cell-steps of a problem (the unit of work of the solver)."""
    return (p.nz + 2 * p.pml) * (p.nx + 2 * p.pml) * p.nt * p.nshot


def schedule(costs, nstreams: int) -> list[list[int]]:
    """Longest-processing-time-first list scheduling of jobs on nstreams
    identical machines; returns the job indices of each stream, in order."""
    if nstreams < 1:
        raise ValueError("nstreams >= 1")
    queues: list[list[int]] = [[] for _ in range(nstreams)]
    load = [0] * nstreams
    for j in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        k = min(range(nstreams), key=lambda s: (load[s], s))
        queues[k].append(j)
        load[k] += costs[j]
    return queues


COHORT = 16  # problems per sweep_gradient_batch call (its launches carry 16 at most)


def cohorts(items: list[Item], size: int = COHORT) -> list[list[int]]:
    """Item indices in groups of `size`, each of similar record length
    (sorted by nt, longest first), so that few problems of a cohort sit idle
    while the others finish their time loop."""
    order = sorted(range(len(items)), key=lambda i: (-items[i].problem.nt, -cost(items[i].problem), i))
    return [order[k:k + size] for k in range(0, len(order), size)]


def run(items: list[Item], mode: int = sweep.MODE_GRADIENT, streams: int = 8,
        device=None, fused: bool = True) -> list[int]:
    """Runs every item; returns the status code of each (0 = ok).  Outputs
    are allocated on first use and written in place.  Acoustic items run as
    cohorts in shared launches unless ``fused`` is False; a batch with an
    elastic item runs one problem per call."""
    device = torch.device(device or "cuda")
    if not items:
        return []
    for it in items:
        gshape, dshape = out_shapes(it.problem)
        if mode == sweep.MODE_GRADIENT:
            if it.grad is None:
                it.grad = torch.empty(gshape, dtype=torch.float32, device=device)
            if it.misfit is None:
                it.misfit = torch.empty((), dtype=torch.float64, device=device)
        elif mode == sweep.MODE_FORWARD and it.data is None:
            it.data = torch.empty(dshape, dtype=torch.float32, device=device)
    codes = torch.zeros(len(items), dtype=torch.int32, device=device)
    errors: list[BaseException] = []
    if any(it.problem.flags & sweep.F_ONE_LAUNCH for it in items):
        # a time-loop launch holds every SM until its loop ends: two of them
        # on different streams would each wait for SMs the other holds
        streams = 1
    if fused and all(it.problem.physics == sweep.ACOUSTIC for it in items):
        groups = cohorts(items)
        gq = [q for q in schedule([sum(cost(items[i].problem) for i in g) for g in groups],
                                  streams) if q]

        def cohort_worker(queue, stream):
            try:
                with torch.cuda.stream(stream):
                    for gi in queue:
                        idx = groups[gi]
                        ws = [sweep.alloc_workspace(items[i].problem, mode, device) for i in idx]
                        common = ([items[i].problem for i in idx], [items[i].model for i in idx],
                                  [items[i].wavelet for i in idx], [items[i].src for i in idx],
                                  [items[i].rec for i in idx])
                        if mode == sweep.MODE_GRADIENT:
                            sweep.sweep_gradient_batch(
                                *common, [items[i].d_obs for i in idx],
                                grads=[items[i].grad for i in idx],
                                misfits=[items[i].misfit for i in idx], ws=ws, stream=stream,
                                sync=False)
                        else:
                            sweep.sweep_forward_batch(*common, data=[items[i].data for i in idx],
                                                      ws=ws, stream=stream, sync=False)
                        for j, i in enumerate(idx):  # the status word leads the workspace
                            codes[i:i + 1].copy_(ws[j][:4].view(torch.int32), non_blocking=True)
            except BaseException as e:  # reported after the join
                errors.append(e)

        return _run_threads(gq, cohort_worker, codes, errors, device)
    queues = [q for q in schedule([cost(it.problem) for it in items], streams) if q]

    def worker(queue, stream):
        try:
            nbytes = max(sweep.workspace_bytes(items[i].problem, mode) for i in queue)
            with torch.cuda.stream(stream):
                ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
                off = (-ws.data_ptr()) % 256
                ws = ws[off:off + nbytes]
                for i in queue:
                    it = items[i]
                    if mode == sweep.MODE_GRADIENT:
                        sweep.sweep_gradient(it.problem, it.model, it.wavelet, it.src, it.rec,
                                             it.d_obs, grad=it.grad, misfit=it.misfit, ws=ws,
                                             stream=stream, sync=False)
                    else:
                        sweep.sweep_forward(it.problem, it.model, it.wavelet, it.src, it.rec,
                                            data=it.data, ws=ws, stream=stream, sync=False)
                    # the status word leads the workspace
                    codes[i:i + 1].copy_(ws[:4].view(torch.int32), non_blocking=True)
        except BaseException as e:  # reported after the join
            errors.append(e)

    return _run_threads(queues, worker, codes, errors, device)


def _run_threads(queues, worker, codes, errors, device) -> list[int]:
    """One stream and one host thread per queue; returns the status codes."""
    pool = [torch.cuda.Stream(device=device) for _ in queues]
    for s in pool:  # inputs made on the current stream are ready first
        s.wait_stream(torch.cuda.current_stream(device))
    threads = [threading.Thread(target=worker, args=(q, s)) for q, s in zip(queues, pool)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for s in pool:
        s.synchronize()
    if errors:
        raise errors[0]
    return [int(c) for c in codes.cpu()]


def tune_key(items: list[Item], candidates, mode: int, fused: bool, device_name: str,
             kind: str = "streams") -> str:
    """Key of a tuning result: what is tuned, the GPU's name, the mode, the
    candidates and every problem's sizes (geometry, border, record length,
    shots, receivers), in order."""
    sig = [device_name, int(mode), bool(fused), [int(c) for c in candidates]]
    if kind != "streams":
        sig.insert(0, kind)
    sig += [[it.problem.physics, it.problem.nz, it.problem.nx, it.problem.pml, it.problem.nt,
             it.problem.nshot, it.problem.nrec] for it in items]
    return hashlib.sha256(json.dumps(sig).encode()).hexdigest()[:32]


def _read_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _write_cache(path: str, key: str, value: dict) -> None:
    d = _read_cache(path)
    d[key] = value
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f)
    os.replace(tmp, path)


def autotune_streams(items: list[Item], candidates=(2, 4, 8, 16),
                     mode: int = sweep.MODE_GRADIENT, device=None, fused: bool = True,
                     cache: str | None = None):
    """Times ``run`` for each stream count; returns (best, {count: seconds}).

    ``cache`` (default: the ``SWEEP_TUNE_CACHE`` environment variable) names
    a JSON file of earlier results: a batch of the same problem sizes on the
    same GPU model with the same candidates takes the stored choice without
    timing anything, and a new result is added to the file (rewritten under
    a temporary name and renamed into place)."""
    cache = cache if cache is not None else os.environ.get("SWEEP_TUNE_CACHE")
    key = None
    if cache:
        dev = torch.device(device or "cuda")
        key = tune_key(items, candidates, mode, fused, torch.cuda.get_device_name(dev))
        hit = _read_cache(cache).get(key)
        if hit is not None:
            return int(hit["best"]), {int(k): float(v) for k, v in hit["seconds"].items()}
    times = {}
    for n in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(items, mode, n, device, fused)
        torch.cuda.synchronize()
        times[n] = time.perf_counter() - t0
    best = min(times, key=lambda n: (times[n], n))
    if key is not None:
        _write_cache(cache, key, {"best": best, "seconds": {str(k): v for k, v in times.items()}})
    return best, times


def stencil_units(p: sweep.Problem) -> int:
    """(tile, shot) work units of a problem's stencil launch in 32-row tiles
    (128-cell wide tiles over the padded grid)."""
    nz, nx = p.nz + 2 * p.pml, p.nx + 2 * p.pml
    return -(-nz // 32) * -(-nx // 128) * p.nshot


def set_tiles(items: list[Item], threshold: int) -> None:
    """16-row stencil tiles for the acoustic problems with fewer than
    `threshold` 32-row units, 32-row tiles for every other problem."""
    for it in items:
        f = it.problem.flags & ~sweep.F_ROWS16
        if it.problem.physics == sweep.ACOUSTIC and stencil_units(it.problem) < threshold:
            f |= sweep.F_ROWS16
        it.problem.flags = f


TILE_THRESHOLDS = (0, 152, 608, 2 ** 31 - 1)  # 0: 32 rows everywhere; max: 16 everywhere


def autotune_tiles(items: list[Item], thresholds=TILE_THRESHOLDS, streams: int = 2,
                   mode: int = sweep.MODE_GRADIENT, device=None, fused: bool = True,
                   cache: str | None = None):
    """Times ``run`` (at `streams` streams) with each threshold of
    ``set_tiles``, leaves the fastest set on the items and returns
    (best threshold, {threshold: seconds}).  Cached like
    ``autotune_streams``."""
    cache = cache if cache is not None else os.environ.get("SWEEP_TUNE_CACHE")
    key = None
    if cache:
        dev = torch.device(device or "cuda")
        key = tune_key(items, list(thresholds) + [streams], mode, fused,
                       torch.cuda.get_device_name(dev), kind="tiles")
        hit = _read_cache(cache).get(key)
        if hit is not None:
            best = int(hit["best"])
            set_tiles(items, best)
            return best, {int(k): float(v) for k, v in hit["seconds"].items()}
    times = {}
    for th in thresholds:
        set_tiles(items, th)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(items, mode, streams, device, fused)
        torch.cuda.synchronize()
        times[int(th)] = time.perf_counter() - t0
    best = min(times, key=lambda t: (times[t], t))
    set_tiles(items, best)
    if key is not None:
        _write_cache(cache, key, {"best": best, "seconds": {str(k): v for k, v in times.items()}})
    return best, times
