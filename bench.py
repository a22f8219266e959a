"""Benchmark of the acoustic forward + adjoint gradient (one JSON line).

Workload: acoustic FWI gradient on a 301 x 901 interior grid (+ 40-cell CPML
per side, 381 x 981 padded), dx = 10 m, dt = 1 ms, nt = 3000, 20 shots at the
surface, 301 receivers every 3 cells, 10 Hz Ricker; the model is the seeded
layered + Gaussian-anomaly starting model, d_obs the forward data of the true
model (synthetic).  One step = one sweep_gradient call: forward with ring
saving, residual + FP64 misfit, backward with reconstruction + imaging, FP64
shot sum; the timed steps replay it from a CUDA graph recorded once
(--no-graph: direct calls).  value = padded cells x nt x shots x ranks / step
time (Gpts/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sweep|reference]

Under torchrun (N > 1) the survey has 20 N surface shots and every rank
models its own contiguous block of 20 of them (weak scaling); the gradients
and misfits are summed over ranks with one all-reduce per step (the shot
sum, the only exchange of the method), which gives the survey's gradient.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_14189_gb300 import inputs  # noqa: E402

METRIC = "Gpts/s fwd+adj"
UNIT = "Gpts/s"
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ac_bwd_marmousi.txt")


def workload_desc(w, nshot):
    return (f"acoustic fwd+adj gradient {w['nz']}x{w['nx']} + {w['pml']}-cell CPML, "
            f"dx {w['dx']:g} m, dt {w['dt'] * 1e3:g} ms, nt {w['nt']}, {nshot} shots, "
            f"{w['rec'].shape[1]} receivers, {w['f0']:g} Hz Ricker")


def counts(nz, nx, P):
    """Cell counts of the padded grid: padded, interior, x-border strip
    cells (2P x NZ), z-border strip cells (2P x NX), saved ring."""
    NZ, NX = nz + 2 * P, nx + 2 * P
    w = min(P, 4)
    return dict(N_pad=NZ * NX, N_int=nz * nx, N_x=2 * P * NZ, N_z=2 * P * NX,
                N_ring=2 * w * (nx + 2 * w) + 2 * nz * w)


def alg_bytes_bwd(c):
    """Algorithmic bytes of one backward step per shot (FP32): reconstruction
    reads u^n, u^{n+1}, K and writes u^{n-1} on the interior; the adjoint
    reads mu^{n+1}, mu^{n+2}, K and writes mu^n on the padded grid (K shared
    with the reconstruction inside); g is read and written on the interior;
    4 adjoint memory variables per border strip cell per axis; ring read."""
    return (20 * c["N_int"] + 16 * c["N_pad"] + 16 * (c["N_x"] + c["N_z"]) + 4 * c["N_ring"])


def alg_bytes_fwd(c):
    return 16 * c["N_pad"] + 16 * (c["N_x"] + c["N_z"]) + 4 * c["N_ring"]


def alg_bytes_k_once(per_shot, c, nshot):
    """Algorithmic bytes of one step of nshot shots when the velocity
    coefficient K (4 B per padded cell, one model for all shots) is counted
    once for the batch instead of once per shot.  The imaging accumulator is
    per shot, so nothing else is shared."""
    return per_shot * nshot - 4 * c["N_pad"] * (nshot - 1)


def interior_gpts(value, c):
    """The throughput in interior cell-steps: the padded figure times the
    interior share of the padded grid."""
    return value * c["N_int"] / c["N_pad"]


# the sources the acoustic time-step kernels are compiled from
KERNEL_SOURCES = ("acoustic_common.cuh", "acoustic_cpml.cu", "acoustic_cpml.cuh",
                  "acoustic_interior.cu", "acoustic_stencil.cuh", "sweep_internal.cuh", "tma.cuh")


def kernel_source_hash():
    """Hash of the time-step kernels' sources with comments and blank space
    removed, so that a profile stays valid across edits that do not change
    the kernels' code."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2604_14189_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in KERNEL_SOURCES:
            src = open(os.path.join(d, f), encoding="utf-8").read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(f.encode() + b"\0" + " ".join(src.split()).encode())
    return h.hexdigest()[:16]


def read_traffic():
    """ncu DRAM bytes per launch of the backward kernel, if the committed
    summary was taken on the current kernel sources."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_hash") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling.  Started before the warm-up so
    that the tool's own start-up (driver initialisation on the host) does not
    overlap the timed region; mark() brackets the timed region, and only the
    samples taken inside it are summarised."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            # one synchronous query first, so that the sampling loop's
            # first sample is not delayed by the tool's own start-up
            subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm",
                            "--format=csv,noheader"], stdout=subprocess.DEVNULL,
                           stderr=subprocess.DEVNULL, timeout=30)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def mark(self):
        """First call: the timed region starts; second call: it ends."""
        import datetime
        now = datetime.datetime.now()
        if self.t0 is None:
            self.t0 = now
        else:
            self.t1 = now

    def stop(self):
        import datetime
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.f.name)

        def when(r):
            try:
                return datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                return None
        if self.t0 is not None and self.t1 is not None:
            lo = self.t0 - datetime.timedelta(seconds=0.25)
            hi = self.t1 + datetime.timedelta(seconds=0.25)
            inside = [r for r in rows if when(r) is not None and lo <= when(r) <= hi]
            rows = inside or rows
        rows = [r[1:] for r in rows]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        loaded = [s for s in sm if smax and s > 0.3 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------- oracle
def oracle_sample(w, nshot_max, nt_sample, threads=None):
    """Time the FP64 oracle gradient on a bounded sample of the workload: the
    same grid and geometry, min(threads, nshot_max) shots, nt_sample steps,
    on `threads` host threads (default: every core)."""
    import oracle
    cores = threads or os.cpu_count() or 1
    ns = max(1, min(nshot_max, cores))
    oracle.set_threads(cores)
    q = oracle.make_problem(0, w["nz"], w["nx"], w["pml"], w["dx"], w["dt"], nt_sample, ns,
                            w["rec"].shape[1], w["f0"])
    wav = np.stack([inputs.ricker(w["f0"], w["dt"], nt_sample)] * ns)
    d_obs = np.zeros((ns, w["rec"].shape[1], nt_sample))
    t = time.perf_counter()
    oracle.acoustic_gradient(q, w["model"], wav, w["src"][:ns], w["rec"][:ns], d_obs)
    el = time.perf_counter() - t
    c = counts(w["nz"], w["nx"], w["pml"])
    gpts = c["N_pad"] * nt_sample * ns / el / 1e9
    return gpts, el, min(ns, cores), (f"oracle gradient, {ns} shots x {nt_sample} steps of the "
                                      f"{w['nz']}x{w['nx']} workload ({el:.1f} s)")


def oracle_fwi_sample(w, nshot_max, nt_sample, grads, forwards):
    """The FP64 oracle's cost of the plain FWI run, from a bounded sample:
    its gradient and its forward modelling timed on min(cores, nshot_max)
    shots x nt_sample steps of the same problem, scaled to `grads` full
    gradients and `forwards` full forward runs (the line-search trials).
    Returns (estimated seconds, sample seconds, cores, description)."""
    import oracle
    cores = os.cpu_count() or 1
    ns = max(1, min(nshot_max, cores))
    oracle.set_threads(cores)
    nrec = w["rec"].shape[1]
    q = oracle.make_problem(0, w["nz"], w["nx"], w["pml"], w["dx"], w["dt"], nt_sample, ns, nrec,
                            w["f0"], v_pml=4500.0)
    wav = np.stack([inputs.ricker(w["f0"], w["dt"], nt_sample)] * ns)
    t = time.perf_counter()
    oracle.acoustic_gradient(q, w["model"], wav, w["src"][:ns], w["rec"][:ns],
                             np.zeros((ns, nrec, nt_sample)))
    tg = time.perf_counter() - t
    t = time.perf_counter()
    oracle.acoustic_forward(q, w["model"], wav, w["src"][:ns], w["rec"][:ns])
    tf = time.perf_counter() - t
    scale = (w["src"].shape[0] / ns) * (w["nt"] / nt_sample)
    est = (grads * tg + forwards * tf) * scale
    return est, tg + tf, ns, (f"oracle gradient ({tg:.1f} s) and forward ({tf:.1f} s) on {ns} "
                              f"shots x {nt_sample} steps of the same problem, scaled to "
                              f"{grads} gradients and {forwards} forward runs of "
                              f"{w['src'].shape[0]} shots x {w['nt']} steps")


def oracle_batch_sample(problems, nt_cap):
    """Time the FP64 oracle gradient of 1/2 |d|^2 on a bounded sample of the
    heterogeneous batch: the given problems, each with its record cut to
    nt_cap steps, run one after another on every core (shots in parallel).
    Returns (padded cell-steps / s in G, seconds, cores, description)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    cells = 0
    t = time.perf_counter()
    for w in problems:
        nt = min(w["nt"], nt_cap)
        ns, nrec = w["src"].shape[0], w["rec"].shape[1]
        q = oracle.make_problem(0, w["nz"], w["nx"], w["pml"], w["dx"], w["dt"], nt, ns, nrec,
                                w["f0"])
        wav = np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * ns)
        oracle.acoustic_gradient(q, w["model"], wav, w["src"], w["rec"],
                                 np.zeros((ns, nrec, nt)))
        cells += (w["nz"] + 2 * w["pml"]) * (w["nx"] + 2 * w["pml"]) * nt * ns
    el = time.perf_counter() - t
    return cells / el / 1e9, el, cores, (f"oracle gradient of the first {len(problems)} "
                                         f"problems, records cut to {nt_cap} steps ({el:.1f} s)")


def run_reference(args, w, rank):
    """Reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    nt_sample = 60
    for _ in range(args.warmup):
        oracle_sample(w, 20, nt_sample)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g, el, cores, sample = oracle_sample(w, 20, nt_sample)
        vals.append(g)
    total = time.perf_counter() - t0
    value = float(np.mean(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w, 20), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------- sweep
def run_sweep(args, w, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2604_14189_gb300 import shots, sweep

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nshot, nt = w["src"].shape[0], w["nt"]
    nrec = w["rec"].shape[1]
    p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                      nshot=nshot, nrec=nrec, f_ref=w["f0"])
    wav_h = np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot).astype(np.float32)
    v0 = torch.tensor(w["model"], dtype=torch.float32, device=dev)
    vt = torch.tensor(w["v_true"], dtype=torch.float32, device=dev)
    wav = torch.tensor(wav_h, device=dev)
    src = torch.tensor(w["src"], device=dev)
    rec = torch.tensor(w["rec"], device=dev)
    d_obs = sweep.sweep_forward(p, vt, wav, src, rec)
    ws = sweep.alloc_workspace(p, sweep.MODE_GRADIENT, dev)
    grad = torch.empty((w["nz"], w["nx"]), dtype=torch.float32, device=dev)
    mis = torch.empty((), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call(st=None):
        sweep.sweep_gradient(p, v0, wav, src, rec, d_obs, grad=grad, misfit=mis, ws=ws,
                             stream=st, sync=False)

    graph = None
    if not args.no_graph:
        # the timed steps replay one recorded sweep_gradient call (same
        # buffers every step); captured on a side stream, replayed on this one
        side = torch.cuda.Stream(dev)
        with sweep.capture(side) as cap:
            call(side)
        graph = cap.graph
        torch.cuda.current_stream(dev).wait_stream(side)

    def step():
        if graph is not None:
            graph.launch(stream)
        else:
            call()
        shots.reduce_gradient(grad, mis)

    def barrier():
        if world > 1:
            dist.barrier()

    sampler = ClockSampler(local_rank)
    sampler.start()  # its start-up overlaps the warm-up, not the timed region
    # The warm-up runs the timed loop's body, L2 flush included: the first
    # launch of torch's fill kernel in a process loads its module (lazy
    # loading), which on a cold page cache stalls the host for ~0.2 s.
    for _ in range(max(args.warmup, 0)):
        flush.zero_()
        step()
    st = sweep.status(ws)
    if st != sweep.OK:
        raise sweep.SweepError(st, "warm-up")

    l0 = sweep.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    sampler.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        if k:
            flush.zero_()  # L2 flush between timed steps (inputs exceed L2 anyway)
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    barrier()
    clocks = sampler.stop()
    launches = sweep.kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    st = sweep.status(ws)
    if st != sweep.OK:
        raise sweep.SweepError(st, "timed region")
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    c = counts(w["nz"], w["nx"], w["pml"])
    pts_step = c["N_pad"] * nt * nshot * world
    value = pts_step / (ms_step * 1e-3) / 1e9

    # per-step kernel durations, on the launching stream, from the same
    # gradient steps again (direct calls: a graph replay records no events):
    # (1) CUDA events before the first and after the last step of each
    # forward and backward time loop, so that consecutive steps keep their
    # programmatic overlap as in the timed region: the step's average
    # duration in the pipeline; (2) events around every step, which end the
    # overlap between steps: each step's duration on its own (reported too)
    prof_steps = max(1, min(args.steps, 2))
    sweep.profile_enable((1 << sweep.K_AC_BWD_LOOP) | (1 << sweep.K_AC_FWD_LOOP))
    for _ in range(prof_steps):
        call()
    torch.cuda.synchronize()
    bwd_loop_ms, bwd_loops = sweep.profile_read(sweep.K_AC_BWD_LOOP)
    fwd_loop_ms, fwd_loops = sweep.profile_read(sweep.K_AC_FWD_LOOP)
    sweep.profile_enable((1 << sweep.K_AC_BWD) | (1 << sweep.K_AC_FWD))
    for _ in range(prof_steps):
        call()
    torch.cuda.synchronize()
    bwd_ms, bwd_n = sweep.profile_read(sweep.K_AC_BWD)
    fwd_ms, fwd_n = sweep.profile_read(sweep.K_AC_FWD)
    sweep.profile_enable(False)

    # end to end through the public API with host buffers
    d_obs_h = d_obs.cpu().pin_memory()
    model_h = torch.tensor(w["model"], dtype=torch.float32).pin_memory()
    wav_hh = torch.tensor(wav_h).pin_memory()
    src_h = torch.tensor(w["src"]).pin_memory()
    rec_h = torch.tensor(w["rec"]).pin_memory()
    grad_h = torch.empty_like(grad, device="cpu").pin_memory()
    mis_h = torch.empty((), dtype=torch.float64).pin_memory()
    bufs = [torch.empty_like(t, device=dev) for t in (model_h, wav_hh, src_h, rec_h, d_obs_h)]
    h2d = sum(t.numel() * t.element_size() for t in (model_h, wav_hh, src_h, rec_h, d_obs_h))
    d2h = grad_h.numel() * grad_h.element_size() + 8

    def e2e_step():
        for dst, srcb in zip(bufs, (model_h, wav_hh, src_h, rec_h, d_obs_h)):
            dst.copy_(srcb, non_blocking=True)
        sweep.sweep_gradient(p, bufs[0], bufs[1], bufs[2], bufs[3], bufs[4], grad=grad,
                             misfit=mis, ws=ws, sync=False)
        shots.reduce_gradient(grad, mis)
        grad_h.copy_(grad, non_blocking=True)
        mis_h.copy_(mis, non_blocking=True)

    e2e_step()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    e2e_value = pts_step / (ms_e2e / args.steps * 1e-3) / 1e9
    if not np.isfinite(float(mis_h)):
        raise RuntimeError("non-finite misfit in the end-to-end run")
    if graph is not None:
        torch.cuda.synchronize()
        graph.close()

    if rank != 0:
        return
    peak, peak_src = peaks()
    # nt + 1 backward steps per loop, of which the first (adjoint only) and
    # the last (imaging only) are partial: the loop's time is divided by the
    # nt - 1 full steps (a slight overestimate of a step's duration)
    bwd_avg_ms = bwd_loop_ms / max(bwd_loops * (nt - 1), 1)
    fwd_avg_ms = fwd_loop_ms / max(fwd_loops * nt, 1)
    bwd_own_ms = bwd_ms / max(bwd_n, 1)
    achieved = alg_bytes_bwd(c) * nshot / (bwd_avg_ms * 1e-3) / 1e9
    traffic = read_traffic()
    path_gbs = (alg_bytes_fwd(c) + alg_bytes_bwd(c)) * nshot * nt / (ms_step * 1e-3) / 1e9
    k_once = alg_bytes_k_once(alg_bytes_bwd(c), c, nshot)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        g, el, cores, sample = oracle_sample(w, nshot, 700)
        g1, _, _, sample1 = oracle_sample(w, 1, 200, threads=1)
        cpu = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": g1, "unit": UNIT, "cores": 1, "sample": sample1}}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc(w, nshot), "nz": w["nz"], "nx": w["nx"],
                   "pml": w["pml"], "nt": nt, "shots_per_gpu": nshot, "nrec": nrec,
                   "l2": "inputs larger than L2 (workspace %.2f GB per step); 256 MB L2 flush "
                         "between timed steps" % (ws.numel() / 1e9),
                   "reductions": "f64",
                   "launch": ("CUDA-graph replay of one recorded sweep_gradient call per step"
                              if graph is not None else "direct sweep_gradient call per step")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "acoustic backward time step: stencil kernel (adjoint, "
                               "reconstruction, imaging) + CPML / receiver / ring kernel",
                     "peak_source": peak_src,
                     "frac_of_8000": achieved / 8000.0,
                     "alg_bytes_per_launch": alg_bytes_bwd(c) * nshot,
                     "avg_launch_ms": bwd_avg_ms,
                     "timing": "CUDA events around each whole backward time loop of %d "
                               "profiled gradient calls after the timed region, divided by "
                               "its nt - 1 full steps (steps keep their programmatic "
                               "overlap)" % prof_steps,
                     "step_alone": {"avg_launch_ms": bwd_own_ms,
                                    "achieved": alg_bytes_bwd(c) * nshot / (bwd_own_ms * 1e-3)
                                    / 1e9,
                                    "frac": alg_bytes_bwd(c) * nshot / (bwd_own_ms * 1e-3)
                                    / 1e9 / peak,
                                    "timing": "CUDA events around every backward step (an "
                                              "event between steps ends their overlap)"}},
        "interior_gpts": interior_gpts(value, c),
        "k_once": {"alg_bytes_per_launch": k_once,
                   "achieved": k_once / (bwd_avg_ms * 1e-3) / 1e9,
                   "frac": k_once / (bwd_avg_ms * 1e-3) / 1e9 / peak,
                   "note": "backward step bytes with K read once for all shots"},
        "path_roofline": {"achieved": path_gbs, "frac": path_gbs / peak,
                          "note": "algorithmic bytes of all forward and backward steps "
                                  "x steps / timed step time"},
        "forward_kernel": {"avg_launch_ms": fwd_avg_ms,
                           "achieved_gbs": alg_bytes_fwd(c) * nshot / (fwd_avg_ms * 1e-3) / 1e9,
                           "step_alone_ms": fwd_ms / max(fwd_n, 1)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if world == 1 and not args.no_extras:
        out["extras"] = run_extras(args, local_rank)
    print(json.dumps(out), flush=True)


# -------------------------------------------------------------------- elastic
def alg_bytes_elastic_fwd(c):
    """Algorithmic bytes of one fused elastic step per shot: 5 fields read and
    written, 5 coefficients read, 4 memory variables read and written per
    strip cell per axis."""
    return 60 * c["N_pad"] + 32 * (c["N_x"] + c["N_z"])


def alg_bytes_elastic_adj(c, nshot):
    """Algorithmic bytes of one fused elastic transposed step per shot: the
    adjoint state (5 fields) read and written, the forward state (5 fields)
    read, the 5 coefficients and the compensated coefficient-adjoint sums
    (5 x hi, lo, read and written) once per step for all shots, 4 adjoint
    memory variables read and written and 4 forward ones read per strip
    cell per axis."""
    return 60 * c["N_pad"] + (20 + 80) * c["N_pad"] / nshot + 48 * (c["N_x"] + c["N_z"])


def run_elastic(args, rank, world, local_rank, emit=True):
    """Elastic forward (isotropic velocity-stress, 500 x 1500 + 40, 64 shots,
    nt 4000, 750 receivers) or elastic gradient (same grid, 8 shots,
    nt = --nt or 1000: the checkpointed replay keeps sqrt(nt) forward
    states per shot in HBM)."""
    import torch

    from paper_2604_14189_gb300 import sweep

    grad_mode = args.workload == "elastic-gradient"
    nshot = 8 if grad_mode else 64
    nt = args.nt if args.nt != 3000 else (1000 if grad_mode else 4000)
    w = inputs.workload_elastic(nshot=nshot, nt=nt)
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nrec = w["rec"].shape[1]
    p = sweep.problem(sweep.ELASTIC, nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"],
                      dt=w["dt"], nt=nt, nshot=nshot, nrec=nrec, f_ref=w["f0"])
    wav_h = np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot).astype(np.float32)
    model = torch.tensor(w["model"], dtype=torch.float32, device=dev)
    wav = torch.tensor(wav_h, device=dev)
    src = torch.tensor(w["src"], device=dev)
    rec = torch.tensor(w["rec"], device=dev)
    stream = torch.cuda.current_stream(dev)
    c = counts(w["nz"], w["nx"], w["pml"])
    if grad_mode:
        m_true = w["model"].copy()
        m_true[:, 150:250, 500:900] *= 1.03
        d_obs = sweep.sweep_forward(p, torch.tensor(m_true, dtype=torch.float32, device=dev),
                                    wav, src, rec)
        ws = sweep.alloc_workspace(p, sweep.MODE_GRADIENT, dev)
        grad = torch.empty((3, w["nz"], w["nx"]), dtype=torch.float32, device=dev)
        mis = torch.empty((), dtype=torch.float64, device=dev)

        def step():
            sweep.sweep_gradient(p, model, wav, src, rec, d_obs, grad=grad, misfit=mis, ws=ws,
                                 sync=False)
    else:
        ws = sweep.alloc_workspace(p, sweep.MODE_FORWARD, dev)
        data = torch.empty((nshot, 2, nrec, nt), dtype=torch.float32, device=dev)

        def step():
            sweep.sweep_forward(p, model, wav, src, rec, data=data, ws=ws, sync=False)

    sampler = ClockSampler(local_rank)
    sampler.start()  # its start-up overlaps the warm-up, not the timed region
    for _ in range(max(args.warmup, 0)):
        step()
    st = sweep.status(ws)
    if st != sweep.OK:
        raise sweep.SweepError(st, "warm-up")
    l0 = sweep.kernel_launches()
    torch.cuda.synchronize()
    sampler.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()  # inputs (4.6 GB of fields per step) exceed L2
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    clocks = sampler.stop()
    launches = sweep.kernel_launches() - l0
    ms_step = e0.elapsed_time(e1) / args.steps
    if sweep.status(ws) != sweep.OK:
        raise sweep.SweepError(sweep.status(ws), "timed region")
    value = c["N_pad"] * nt * nshot / (ms_step * 1e-3) / 1e9
    # per-step kernel time of the forward (velocity + stress kernels) and,
    # for the gradient, of the transposed step
    sweep.profile_enable((1 << sweep.K_EL_VEL) | (1 << sweep.K_EL_STR) |
                         (1 << sweep.K_EL_ADJ))
    step()
    torch.cuda.synchronize()
    vms, vn = sweep.profile_read(sweep.K_EL_VEL)
    sms, sn = sweep.profile_read(sweep.K_EL_STR)
    ams, an = sweep.profile_read(sweep.K_EL_ADJ)
    sweep.profile_enable(False)
    step_ms = vms / max(vn, 1) + sms / max(sn, 1)
    adj_ms = ams / max(an, 1)
    adj_bytes = alg_bytes_elastic_adj(c, nshot) * nshot
    peak, peak_src = peaks()
    achieved = alg_bytes_elastic_fwd(c) * nshot / (step_ms * 1e-3) / 1e9
    # end to end with host buffers
    model_h = torch.tensor(w["model"], dtype=torch.float32).pin_memory()
    wav_hh = torch.tensor(wav_h).pin_memory()
    if grad_mode:
        dob_h = d_obs.cpu().pin_memory()
        grad_h = torch.empty_like(grad, device="cpu").pin_memory()
        bufs = [torch.empty_like(t, device=dev) for t in (model_h, wav_hh, dob_h)]
        h2d = sum(t.numel() * t.element_size() for t in (model_h, wav_hh, dob_h))
        d2h = grad_h.numel() * 4 + 8

        def e2e():
            for dst, sb in zip(bufs, (model_h, wav_hh, dob_h)):
                dst.copy_(sb, non_blocking=True)
            sweep.sweep_gradient(p, bufs[0], bufs[1], src, rec, bufs[2], grad=grad, misfit=mis,
                                 ws=ws, sync=False)
            grad_h.copy_(grad, non_blocking=True)
    else:
        data_h = torch.empty_like(data, device="cpu").pin_memory()
        bufs = [torch.empty_like(t, device=dev) for t in (model_h, wav_hh)]
        h2d = sum(t.numel() * t.element_size() for t in (model_h, wav_hh))
        d2h = data_h.numel() * 4

        def e2e():
            for dst, sb in zip(bufs, (model_h, wav_hh)):
                dst.copy_(sb, non_blocking=True)
            sweep.sweep_forward(p, bufs[0], bufs[1], src, rec, data=data, ws=ws, sync=False)
            data_h.copy_(data, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    e2e()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = c["N_pad"] * nt * nshot / (e0.elapsed_time(e1) * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        oracle.set_threads(cores)
        ns_s, nt_s = (2, 30) if grad_mode else (4, 30)
        q = oracle.make_problem(1, w["nz"], w["nx"], w["pml"], w["dx"], w["dt"], nt_s, ns_s,
                                nrec, w["f0"], v_pml=5000.0)
        wv = np.stack([inputs.ricker(w["f0"], w["dt"], nt_s)] * ns_s)
        t = time.perf_counter()
        if grad_mode:
            oracle.elastic_gradient(q, w["model"], wv, w["src"][:ns_s], w["rec"][:ns_s],
                                    np.zeros((ns_s, 2, nrec, nt_s)))
        else:
            oracle.elastic_forward(q, w["model"], wv, w["src"][:ns_s], w["rec"][:ns_s])
        el = time.perf_counter() - t
        cpu = {"value": c["N_pad"] * nt_s * ns_s / el / 1e9, "unit": "Gpts/s",
               "cores": min(cores, ns_s), "kind": "oracle",
               "sample": f"oracle elastic {'gradient' if grad_mode else 'forward'}, "
                         f"{ns_s} shots x {nt_s} steps of the same grid ({el:.1f} s)"}
    metric = "Gpts/s elastic fwd+adj" if grad_mode else "Gpts/s elastic fwd"
    out = {
        "metric": metric, "value": value, "unit": "Gpts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"elastic {'gradient' if grad_mode else 'forward'} "
                               f"{w['nz']}x{w['nx']} + {w['pml']}-cell CPML, dx 5 m, dt 0.5 ms, "
                               f"nt {nt}, {nshot} shots, {nrec} receivers (vx, vz), 15 Hz "
                               f"explosive Ricker",
                   "l2": "fields of all shots (%.1f GB) exceed L2" % (ws.numel() / 1e9)},
        "roofline": ({"bound": "hbm", "achieved": adj_bytes / (adj_ms * 1e-3) / 1e9,
                      "peak": peak, "unit": "GB/s",
                      "frac": adj_bytes / (adj_ms * 1e-3) / 1e9 / peak, "traffic": None,
                      "kernel": "elastic transposed step (stress half, receiver injection, "
                                "velocity half)",
                      "peak_source": peak_src, "alg_bytes_per_launch": adj_bytes,
                      "avg_launch_ms": adj_ms,
                      "timing": "CUDA events around every transposed step of one profiled "
                                "gradient after the timed region"}
                     if grad_mode else
                     {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                      "frac": achieved / peak, "traffic": None,
                      "kernel": "elastic forward step (velocity + stress kernels)",
                      "peak_source": peak_src,
                      "alg_bytes_per_launch": alg_bytes_elastic_fwd(c) * nshot,
                      "avg_launch_ms": step_ms}),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "Gpts/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if grad_mode:
        # the whole gradient in fused algorithmic bytes: the forward pass, the
        # replay and the transposed steps
        path = nt * (2 * alg_bytes_elastic_fwd(c) * nshot + adj_bytes)
        out["path_roofline"] = {"achieved": path / (ms_step * 1e-3) / 1e9,
                                "frac": path / (ms_step * 1e-3) / 1e9 / peak,
                                "note": "fused algorithmic bytes of the forward pass, the "
                                        "replay and the transposed steps / timed gradient"}
        out["forward_kernel"] = {"avg_launch_ms": step_ms, "achieved_gbs": achieved}
    if emit and rank == 0:
        print(json.dumps(out), flush=True)
    return out


# ------------------------------------------------------------------------ fwi
def run_fwi(args, local_rank, emit=True):
    """Plain (illumination-preconditioned) FWI: 20 iterations on the seeded
    256 x 256 layered + anomaly model, 16 shots, nt 1500.  The relative model
    error after 20 plain iterations is the target error of the comparison
    with a learned preconditioner; value = seconds to reach it."""
    import torch

    from paper_2604_14189_gb300 import fwi, sweep

    w = inputs.workload_fwi()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nshot, nt, nrec = w["src"].shape[0], w["nt"], w["rec"].shape[1]
    p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                      nshot=nshot, nrec=nrec, f_ref=w["f0"], v_pml=4500.0)
    wav = torch.tensor(np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot),
                       dtype=torch.float32, device=dev)
    src = torch.tensor(w["src"], device=dev)
    rec = torch.tensor(w["rec"], device=dev)
    vt = torch.tensor(w["v_true"], dtype=torch.float32, device=dev)
    d_obs = sweep.sweep_forward(p, vt, wav, src, rec)
    inv = fwi.Fwi(p, wav, src, rec, d_obs)
    m0 = torch.tensor(w["model"], dtype=torch.float32, device=dev)
    cfg = fwi.FwiConfig(iterations=20, step=50.0, vmin=1400.0, vmax=4700.0)
    sampler = ClockSampler(local_rank)
    sampler.start()  # its start-up overlaps the warm-up, not the timed region
    for _ in range(max(args.warmup, 0)):
        inv.gradient(m0)
        inv.misfit(m0)
    l0 = sweep.kernel_launches()
    torch.cuda.synchronize()
    sampler.mark()
    t0 = time.perf_counter()
    model, hist = inv.run(m0, cfg)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    sampler.mark()
    clocks = sampler.stop()
    launches = sweep.kernel_launches() - l0
    e0 = float((m0 - vt).norm() / vt.norm())
    e1 = float((model - vt).norm() / vt.norm())
    # end to end: the starting model, the observed data and the wavelets
    # copied from pinned host memory into the loop's buffers, the final model
    # copied back, in a second timed run
    m0_h, do_h, wav_h = (t.cpu().pin_memory() for t in (m0, d_obs, wav))
    out_h = torch.empty(m0.shape, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m0_d = m0_h.to(dev, non_blocking=True)
    d_obs.copy_(do_h, non_blocking=True)  # the buffers the recorded graphs read
    wav.copy_(wav_h, non_blocking=True)
    model_e2e, _ = inv.run(m0_d, cfg)
    out_h.copy_(model_e2e, non_blocking=True)
    torch.cuda.synchronize()
    seconds_e2e = time.perf_counter() - t0
    h2d = sum(t.numel() * t.element_size() for t in (m0_h, do_h, wav_h))
    c = counts(w["nz"], w["nx"], w["pml"])
    # the backward time loop timed as a whole (events before its first and
    # after its last step), divided by its nt - 1 full steps
    sweep.profile_enable(1 << sweep.K_AC_BWD_LOOP)
    sweep.sweep_gradient(p, model.contiguous(), wav, src, rec, d_obs, want_illum=True,
                         ws=inv.ws_g)  # a direct call: graph replays record no events
    torch.cuda.synchronize()
    inv.close()
    bms, bn = sweep.profile_read(sweep.K_AC_BWD_LOOP)
    bn *= nt - 1
    sweep.profile_enable(False)
    peak, peak_src = peaks()
    achieved = alg_bytes_bwd(c) * nshot / (bms / max(bn, 1) * 1e-3) / 1e9
    grads = len(hist)
    trials = sum(h["trials"] for h in hist)
    cpu = None
    if not args.no_cpu_baseline:
        est, el, cores, sample = oracle_fwi_sample(w, 16, 200, grads, trials)
        cpu = {"value": est, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample}
    out = {
        "metric": "FWI s to target model error (plain)", "value": seconds, "unit": "s",
        "n_gpus": 1, "steps": grads, "warmup": args.warmup,
        "ms_per_step": seconds * 1e3 / max(grads, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plain illumination-preconditioned FWI, 20 iterations, "
                               f"{w['nz']}x{w['nx']} + {w['pml']}-cell CPML, dx 10 m, nt {nt}, "
                               f"{nshot} shots, {nrec} receivers, 10 Hz",
                   "model_error_initial": e0, "model_error_final": e1,
                   "misfit_initial": hist[0]["misfit"], "misfit_final": hist[-1]["misfit_after"],
                   "gradients": grads, "line_search_forwards": trials,
                   "step": "a gradient (step) plus its line-search forwards",
                   "launch": "recorded CUDA graphs replayed per evaluation (gradient; "
                             "forward + two FP64 dot products)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "acoustic backward time step (as in the headline workload)",
                     "peak_source": peak_src, "avg_launch_ms": bms / max(bn, 1)},
        "cpu_baseline": cpu,
        "e2e": {"value": seconds_e2e, "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": out_h.numel() * 4},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if emit:
        print(json.dumps(out), flush=True)
    return out


# -------------------------------------------------------- learned preconditioner
UNET_LAYERS = [  # (level, cin, cout) of the 17 convolutions, forward order
    (1, 32, 32), (1, 32, 32), (2, 32, 64), (2, 64, 64), (3, 64, 128), (3, 128, 128),
    (4, 128, 256), (4, 256, 256), (3, 256, 128), (3, 256, 128), (3, 128, 128),
    (2, 128, 64), (2, 128, 64), (2, 64, 64), (1, 64, 32), (1, 64, 32), (1, 32, 32)]


def unet_conv_flops(B, H, W, training):
    """FLOPs (2 per multiply-add) of the U-Net's 3 x 3 convolutions: one
    forward pass, or a training step (forward, data gradients of every layer
    but the first, weight gradients)."""
    f = [2.0 * B * (H >> (lv - 1)) * (W >> (lv - 1)) * 9 * ci * co for lv, ci, co in UNET_LAYERS]
    return sum(f) * 3 - f[0] if training else sum(f)


def bf16_peaks():
    try:
        m = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(m["bf16_tflops"]), float(m["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "fallback"


def time_conv(unet, B, H, W, cin, cout, reps=30):
    """Average device time (ms) of one tensor-core convolution launch on
    the launching stream (CUDA events), inputs resident."""
    import ctypes

    import torch
    x = torch.randn((B, H, W, cin), device="cuda").to(torch.bfloat16)
    w = (torch.randn((cout, 9, cin), device="cuda") * (2.0 / (9 * cin)) ** 0.5).to(torch.bfloat16)
    b = torch.zeros(cout, device="cuda")
    out = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()

    def call():
        rc = unet._lib.sweep_unet_conv3x3(B, H, W, cin, cout, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(w.data_ptr()),
                                          ctypes.c_void_p(b.data_ptr()), unet.OP_RELU, None,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(ws.data_ptr()), 256,
                                          ctypes.c_void_p(st.cuda_stream))
        assert rc == 0
    for _ in range(3):
        call()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        call()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def time_train_steps(unet, precond, B, n, steps, warmup):
    """Average wall time (ms) of one U-Net training step (gradient + Adam),
    batch B of n x n two-channel images resident on the GPU."""
    import torch
    s = unet.shape(B, n, n, 2)
    th = precond.init_params(0)
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    x = torch.randn(B, n, n, 2, device="cuda")
    t = torch.randn(B, n, n, device="cuda") * 0.1
    ws = unet.alloc_workspace(s, True)
    grad = torch.empty_like(th)
    out = torch.empty((B, n, n), device="cuda")
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    k = 0
    for _ in range(warmup):
        k += 1
        unet.gradient(s, th, x, t, grad=grad, out=out, loss=loss, ws=ws, sync=False)
        unet.adam(th, grad, m, v, k, 1e-4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        k += 1
        unet.gradient(s, th, x, t, grad=grad, out=out, loss=loss, ws=ws, sync=False)
        unet.adam(th, grad, m, v, k, 1e-4)
    e1.record()
    torch.cuda.synchronize()
    if sweep_status_of(ws) != 0:
        raise RuntimeError("unet training step reported an error")
    return e0.elapsed_time(e1) / steps


def sweep_status_of(ws):
    from paper_2604_14189_gb300 import sweep
    return sweep.status(ws)


def run_unet(args, local_rank):
    """The U-Net's tensor-core kernels alone: --workload unet-conv times one
    3 x 3 convolution launch (--conv B,H,W,cin,cout) against the burst BF16
    peak; --workload unet-train times training steps of batch 8 on 256 x 256
    images against the sustained peak."""
    import torch

    from paper_2604_14189_gb300 import precond, sweep, unet
    torch.cuda.set_device(local_rank)
    burst, sustained, psrc = bf16_peaks()
    l0 = sweep.kernel_launches()
    if args.workload == "unet-conv":
        B, H, W, ci, co = (int(v) for v in args.conv.split(","))
        ms = time_conv(unet, B, H, W, ci, co, reps=max(args.steps, 1))
        flops = 2.0 * B * H * W * 9 * ci * co
        val = flops / (ms * 1e-3) / 1e12
        desc = f"3x3 convolution {ci}->{co} channels on {B} x {H} x {W} (BF16, FP32 accumulation)"
        peak, note = burst, "burst"
    else:
        ms = time_train_steps(unet, precond, 8, 256, max(args.steps, 1), max(args.warmup, 1))
        val = unet_conv_flops(8, 256, 256, True) / (ms * 1e-3) / 1e12
        desc = "U-Net training step (forward, backward, Adam), batch 8 of 256 x 256 x 2"
        peak, note = sustained, "sustained"
    out = {"metric": "TFLOP/s (3x3 convolution FLOPs)", "value": val, "unit": "TFLOP/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic", "config": {"workload": desc},
           "roofline": {"bound": "tensor", "achieved": val, "peak": peak, "unit": "TFLOP/s",
                        "frac": val / peak, "traffic": None, "peak_source": f"{psrc} ({note})"},
           "cpu_baseline": None,
           "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "gpu_launches": int(sweep.kernel_launches() - l0)}
    print(json.dumps(out), flush=True)


def oracle_unet_sample(n=256):
    """The FP64 oracle's U-Net training step (forward + backward) on one
    n x n two-channel image: seconds per image on the host cores."""
    from oracle import unet as U
    rng = np.random.default_rng(0)
    theta = U.init_params(0)
    x = rng.standard_normal((1, n, n, 2))
    t = rng.standard_normal((1, n, n))
    t0 = time.perf_counter()
    U.loss_and_grad(theta, x, t, rounding=True)
    return time.perf_counter() - t0


def run_fwi_learned(args, local_rank):
    """Learned gradient preconditioner: training pairs from the solver
    (seeded 256 x 256 layered + anomaly models, 16 shots, nt 1500), U-Net
    training on the tensor cores, then 20-iteration FWI on held-out seeded
    models, plain (illumination-preconditioned) against learned (gated by
    the plain direction and the solver's misfit, plain fallback).  value =
    median over the held-out models of the learned run's wall seconds to
    reach the plain run's 20-iteration model error."""
    import torch

    from paper_2604_14189_gb300 import fwi, precond, sweep, unet

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n, nshot, nt = 256, 16, 1500
    # 1. pairs
    pairs = precond.generate_pairs(args.pairs, seed=200000, n=n, nshot=nshot, nt=nt,
                                   device=dev)
    # 2. training
    tr = precond.train(pairs.inputs, pairs.targets, epochs=args.epochs, batch=8, lr=1e-3,
                       seed=1)
    step_flops = unet_conv_flops(8, n, n, True)
    train_tflops = step_flops * tr.steps / tr.seconds / 1e12
    # 3. the tensor-core convolution in isolation (the largest-N layer at
    # level 3: 256 -> 128 channels on 64 x 64, batch 8), and a level-1 layer
    t_dec3a = time_conv(unet, 8, 64, 64, 256, 128)
    f_dec3a = 2.0 * 8 * 64 * 64 * 9 * 256 * 128
    t_enc1b = time_conv(unet, 8, 256, 256, 32, 32)
    f_enc1b = 2.0 * 8 * 256 * 256 * 9 * 32 * 32
    t_bot = time_conv(unet, 8, 32, 32, 256, 256)
    f_bot = 2.0 * 8 * 32 * 32 * 9 * 256 * 256
    # 4. held-out FWI, plain vs learned
    p, wav, src, rec = precond.solver_setup(n, nshot, nt, dev)
    cfg = fwi.FwiConfig(iterations=20, step=50.0, vmin=1400.0, vmax=4700.0)
    pre = precond.Preconditioner(tr.theta, n)
    rows = []
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = sweep.kernel_launches()
    models = list(inputs.precond_heldout(args.heldout + 1, seed=900000, n=n))
    for k, (vt_np, v0_np) in enumerate(models):
        vt = torch.tensor(vt_np, dtype=torch.float32, device=dev)
        v0 = torch.tensor(v0_np, dtype=torch.float32, device=dev)
        d_obs = sweep.sweep_forward(p, vt, wav, src, rec)
        inv = fwi.Fwi(p, wav, src, rec, d_obs)
        if k == 0:  # warm-up run (graphs, lazy loading), not reported
            precond.run_plain(inv, v0, fwi.FwiConfig(iterations=2, step=50.0, vmin=1400.0,
                                                     vmax=4700.0), vt)
            precond.run_learned(inv, pre, v0, fwi.FwiConfig(iterations=2, step=50.0,
                                                            vmin=1400.0, vmax=4700.0), vt)
            inv.close()
            sampler.mark()
            continue
        torch.cuda.synchronize()
        _, hp = precond.run_plain(inv, v0, cfg, vt)
        target = hp[-1]["model_error"]  # the plain method's 20-iteration error
        tp = precond.seconds_to(hp, target)
        # up to twice the plain run's iterations, to time the learned run to
        # the target even where it needs more iterations than the plain one
        cfg_l = fwi.FwiConfig(iterations=2 * cfg.iterations, step=cfg.step, vmin=cfg.vmin,
                              vmax=cfg.vmax)
        _, hl = precond.run_learned(inv, pre, v0, cfg_l, vt, cos_min=args.cos_min,
                                    target_error=target)
        tl = precond.seconds_to(hl, target)
        inv.close()
        rows.append(dict(e0=precond.model_error(v0, vt), target=target, plain_s=tp,
                         learned_s=tl, plain_iters=len(hp), learned_iters=len(hl),
                         learned_used=sum(h["used"] == "learned" for h in hl),
                         cos_mean=float(np.nanmean([h["cosine"] for h in hl]))))
    torch.cuda.synchronize()
    sampler.mark()
    clocks = sampler.stop()
    launches = sweep.kernel_launches() - l0
    reached = [r for r in rows if r["learned_s"] is not None]
    lsec = [r["learned_s"] for r in reached]
    psec = [r["plain_s"] for r in rows]
    speed = [r["plain_s"] / r["learned_s"] for r in reached]
    burst, sustained, psrc = bf16_peaks()
    ach = f_dec3a / (t_dec3a * 1e-3) / 1e12
    cpu_s = oracle_unet_sample(n) if not args.no_cpu_baseline else None
    out = {
        "metric": "FWI s to target model error (learned vs plain)",
        "value": statistics.median(lsec) if lsec else None, "unit": "s",
        "n_gpus": 1, "steps": len(rows), "warmup": 1,
        "ms_per_step": 1e3 * statistics.median(lsec) if lsec else None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {
            "workload": f"learned U-Net gradient preconditioner: {args.pairs} solver-generated "
                        f"pairs on seeded {n}x{n} layered + anomaly models (16 shots, nt {nt}, "
                        f"dx 10 m), {args.epochs} epochs, then 20-iteration FWI on "
                        f"{len(rows)} held-out models, plain vs learned",
            "target": "each held-out model's plain 20-iteration relative model error "
                      "(starting model: the true one blurred by a 20-cell Gaussian)",
            "plain_s_median": statistics.median(psec) if psec else None,
            "learned_s_median": statistics.median(lsec) if lsec else None,
            "learned_reached_target": f"{len(reached)}/{len(rows)}",
            "speedup_median": statistics.median(speed) if speed else None,
            "learned_steps_used": sum(r["learned_used"] for r in rows),
            "iterations_total": sum(r["learned_iters"] for r in rows),
            "cosine_mean": float(np.mean([r["cos_mean"] for r in rows])) if rows else None,
            "pairs_seconds": pairs.seconds,
            "pairs_gpts_fwd_adj": pairs.cell_steps / pairs.seconds / 1e9,
            "train_seconds": tr.seconds, "train_steps": tr.steps,
            "train_loss_final": tr.epochs[-1]["train_loss"] if tr.epochs else None,
            "val_loss_first": tr.epochs[0]["val_loss"] if tr.epochs else None,
            "val_loss_final": tr.epochs[-1]["val_loss"] if tr.epochs else None,
            "per_model": rows,
        },
        "roofline": {"bound": "tensor", "achieved": ach, "peak": burst, "unit": "TFLOP/s",
                     "frac": ach / burst, "traffic": None, "peak_source": psrc,
                     "kernel": "conv_kernel (tcgen05 implicit GEMM), 3x3 256->128 channels "
                               "on 8 x 64 x 64, timed alone (burst peak)",
                     "avg_launch_ms": t_dec3a},
        "other_convs": {
            "3x3 32->32 on 8 x 256 x 256": {"ms": t_enc1b,
                                            "tflops": f_enc1b / (t_enc1b * 1e-3) / 1e12},
            "3x3 256->256 on 8 x 32 x 32": {"ms": t_bot,
                                            "tflops": f_bot / (t_bot * 1e-3) / 1e12}},
        "training_roofline": {"achieved": train_tflops, "peak": sustained, "unit": "TFLOP/s",
                              "frac": train_tflops / sustained,
                              "note": "3x3 convolution FLOPs of a batch-8 training step "
                                      "(forward, data and weight gradients) x steps / "
                                      "training wall time (sustained peak)"},
        "cpu_baseline": None if cpu_s is None else {
            "value": cpu_s, "unit": "s per 256x256 training sample", "cores": os.cpu_count(),
            "kind": "oracle", "sample": "FP64 numpy U-Net forward + backward, one image"},
        "e2e": {"value": statistics.median(lsec) if lsec else None, "unit": "s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------- batch
def run_batch(args, local_rank, emit=True):
    """Heterogeneous batch: 256 seeded layered models of uneven size, border,
    record length and shot count, forward + adjoint gradient of 1/2 |d|^2
    each, run concurrently (batch.run); value = padded cell-steps of the
    whole batch / wall time."""
    import torch

    from paper_2604_14189_gb300 import batch, sweep

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    items = []
    cells = alg = alg_b = 0
    problems = inputs.workload_batch()
    for w in problems:
        ns, nrec, nt = w["src"].shape[0], w["rec"].shape[1], w["nt"]
        p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                          nshot=ns, nrec=nrec, f_ref=w["f0"])
        items.append(batch.Item(
            p, torch.tensor(w["model"], dtype=torch.float32, device=dev),
            torch.tensor(np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * ns),
                         dtype=torch.float32, device=dev),
            torch.tensor(w["src"], device=dev), torch.tensor(w["rec"], device=dev),
            d_obs=torch.zeros((ns, 1, nrec, nt), dtype=torch.float32, device=dev)))
        cells += batch.cost(p)
        cb = counts(w["nz"], w["nx"], w["pml"])
        alg += (alg_bytes_fwd(cb) + alg_bytes_bwd(cb)) * ns * nt
        alg_b += alg_bytes_bwd(cb) * ns * nt
    # schedule and tile-height autotuning on a sample of the batch; the
    # tile threshold chosen on the sample is applied to every problem
    best, times = batch.autotune_streams(items[:64], candidates=(1, 2, 3, 4, 6))
    tile_th, tile_times = batch.autotune_tiles(items[:64], streams=best)
    batch.set_tiles(items, tile_th)
    sampler = ClockSampler(local_rank)
    sampler.start()  # its start-up overlaps the warm-up, not the timed region
    for _ in range(max(args.warmup, 0)):
        batch.run(items, streams=best)
    l0 = sweep.kernel_launches()
    torch.cuda.synchronize()
    sampler.mark()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        codes = batch.run(items, streams=best)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / args.steps
    sampler.mark()
    clocks = sampler.stop()
    launches = sweep.kernel_launches() - l0
    if any(codes):
        raise RuntimeError(f"batch errors: {sorted(set(codes))}")
    value = cells / sec / 1e9

    # the dominant kernels: every cohort's backward time loop (stencil + CPML
    # launches of up to 16 problems per step) timed as a whole with CUDA
    # events on its stream, one more pass at one stream so that the loops do
    # not share the GPU with each other
    sweep.profile_enable((1 << sweep.K_AC_BWD_LOOP) | (1 << sweep.K_AC_FWD_LOOP))
    batch.run(items, streams=1)
    torch.cuda.synchronize()
    bwd_loop_ms, bwd_loops = sweep.profile_read(sweep.K_AC_BWD_LOOP)
    fwd_loop_ms, _ = sweep.profile_read(sweep.K_AC_FWD_LOOP)
    sweep.profile_enable(False)
    cohort_steps = sum(max(items[i].problem.nt for i in g) + 1 for g in batch.cohorts(items))
    peak, peak_src = peaks()
    b_gbs = alg_b / (bwd_loop_ms * 1e-3) / 1e9

    # end to end: every problem's model, wavelets, geometry and observed data
    # copied from pinned host memory, and its gradient and misfit copied back,
    # inside the timed pass
    host = [tuple(t.cpu().pin_memory() for t in (it.model, it.wavelet, it.src, it.rec, it.d_obs))
            for it in items]
    h2d = sum(t.numel() * t.element_size() for h in host for t in h)
    g_host = [torch.empty(it.grad.shape, dtype=torch.float32).pin_memory() for it in items]
    m_host = torch.empty(len(items), dtype=torch.float64).pin_memory()
    d2h = sum(g.numel() * 4 for g in g_host) + 8 * len(items)

    def e2e_pass():
        for it, h in zip(items, host):
            for dst, src_h in zip((it.model, it.wavelet, it.src, it.rec, it.d_obs), h):
                dst.copy_(src_h, non_blocking=True)
        c = batch.run(items, streams=best)
        for it, gh in zip(items, g_host):
            gh.copy_(it.grad, non_blocking=True)
        m_host.copy_(torch.stack([it.misfit for it in items]), non_blocking=True)
        torch.cuda.synchronize()
        return c

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    codes = e2e_pass()
    sec_e2e = time.perf_counter() - t0
    if any(codes) or not np.isfinite(m_host.numpy()).all():
        raise RuntimeError("batch end-to-end pass failed")
    cpu = None
    if not args.no_cpu_baseline:
        g, _, cores, sample = oracle_batch_sample(problems[:16], 60)
        cpu = {"value": g, "unit": "Gpts/s", "cores": cores, "kind": "oracle", "sample": sample}
    out = {
        "metric": "Gpts/s fwd+adj (heterogeneous batch)", "value": value, "unit": "Gpts/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "256 seeded layered models, interior 128..512 squared (uneven), "
                               "20..40-cell CPML, nt 800..3000, 1..8 shots, gradient of "
                               "1/2 |d|^2 each", "padded_cell_steps": cells,
                   "streams": best, "autotune_seconds": times,
                   "rows16_below_units": tile_th, "tile_autotune_seconds": tile_times,
                   "step": "one pass over the whole batch"},
        "roofline": {"bound": "hbm", "achieved": b_gbs, "peak": peak, "unit": "GB/s",
                     "frac": b_gbs / peak, "traffic": None,
                     "kernel": "acoustic backward time steps of the cohorts (stencil + CPML "
                               "launches carrying up to 16 problems' steps)",
                     "peak_source": peak_src,
                     "alg_bytes_per_launch": alg_b / cohort_steps,
                     "avg_launch_ms": bwd_loop_ms / cohort_steps,
                     "timing": "CUDA events around every cohort's whole backward time loop "
                               "(%d loops, %d cohort steps) in a pass at one stream after the "
                               "timed region" % (bwd_loops, cohort_steps),
                     "forward_loops_ms": fwd_loop_ms},
        "path_roofline": {"achieved": alg / sec / 1e9, "frac": alg / sec / 1e9 / peak,
                          "note": "algorithmic bytes of every forward and backward step of "
                                  "the 256 problems / pass time"},
        "cpu_baseline": cpu,
        "e2e": {"value": cells / sec_e2e / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if emit:
        print(json.dumps(out), flush=True)
    return out


# --------------------------------------------------------------------- extras
def run_forward200(args, local_rank, emit=True):
    """Single-shot acoustic forward on the 200 x 200 three-layer model (+40
    CPML, nt 1000, 200 receivers): microseconds per time step, replayed from
    a recorded graph (one call per run)."""
    import torch

    from paper_2604_14189_gb300 import sweep
    w = inputs.workload_layered3()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nt, nrec = w["nt"], w["rec"].shape[1]
    p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                      nshot=1, nrec=nrec, f_ref=w["f0"])
    model = torch.tensor(w["model"], dtype=torch.float32, device=dev)
    wav_h = inputs.ricker(w["f0"], w["dt"], nt)[None].astype(np.float32)
    wav = torch.tensor(wav_h, device=dev)
    src = torch.tensor(w["src"], device=dev)
    rec = torch.tensor(w["rec"], device=dev)
    ws = sweep.alloc_workspace(p, sweep.MODE_FORWARD, dev)
    data = torch.empty((1, 1, nrec, nt), dtype=torch.float32, device=dev)
    side = torch.cuda.Stream(dev)
    with sweep.capture(side) as cap:
        sweep.sweep_forward(p, model, wav, src, rec, data=data, ws=ws, stream=side)
    torch.cuda.current_stream(dev).wait_stream(side)
    graph, stream = cap.graph, torch.cuda.current_stream(dev)
    runs = max(args.steps, 1) * 4
    sampler = ClockSampler(local_rank)
    sampler.start()  # its start-up overlaps the warm-up, not the timed region
    for _ in range(max(args.warmup, 1)):
        graph.launch(stream)
    l0 = sweep.kernel_launches()
    torch.cuda.synchronize()
    sampler.mark()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(runs):
        graph.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    clocks = sampler.stop()
    launches = sweep.kernel_launches() - l0
    if sweep.status(ws) != sweep.OK:
        raise sweep.SweepError(sweep.status(ws), "forward 200")
    ms_run = e0.elapsed_time(e1) / runs
    c = counts(w["nz"], w["nx"], w["pml"])
    peak, psrc = peaks()
    # end to end: model and wavelet from pinned host memory, record back
    mh = torch.tensor(w["model"], dtype=torch.float32).pin_memory()
    whh = torch.tensor(wav_h).pin_memory()
    dh = torch.empty((1, 1, nrec, nt), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(runs):
        model.copy_(mh, non_blocking=True)
        wav.copy_(whh, non_blocking=True)
        graph.launch(stream)
        dh.copy_(data, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / runs
    graph.close()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        q = oracle.make_problem(0, w["nz"], w["nx"], w["pml"], w["dx"], w["dt"], 200, 1, nrec,
                                w["f0"])
        oracle.set_threads(1)
        t = time.perf_counter()
        oracle.acoustic_forward(q, w["model"], wav_h[:, :200].astype(np.float64), w["src"],
                                w["rec"])
        el = time.perf_counter() - t
        cpu = {"value": el / 200 * 1e6, "unit": "us per step", "cores": 1, "kind": "oracle",
               "sample": f"oracle forward, 200 of the 1000 steps ({el:.2f} s)"}
    us = ms_run * 1e3 / nt
    out = {"metric": "us per time step (single-shot forward)", "value": us,
           "unit": "us/step", "higher_is_better": False, "ms_per_step": ms_run,
           "config": {"workload": "acoustic forward, 200x200 + 40-cell CPML, nt 1000, 1 shot, "
                                  "200 receivers, three-layer 1500/2500/3500 m/s",
                      "launch": "CUDA-graph replay of one recorded sweep_forward call",
                      "l2": "working set L2-resident (launch-bound size)"},
           "path_roofline": {"achieved": alg_bytes_fwd(c) / (us * 1e-6) / 1e9,
                             "frac": alg_bytes_fwd(c) / (us * 1e-6) / 1e9 / peak,
                             "note": "algorithmic bytes of a forward step / step time (the "
                                     "data stay in L2, so this can pass the HBM peak)"},
           "cpu_baseline": cpu,
           "e2e": {"value": ms_e2e * 1e3 / nt, "unit": "us/step",
                   "h2d_bytes_per_step": (mh.numel() + whh.numel()) * 4 // nt,
                   "d2h_bytes_per_step": dh.numel() * 4 // nt},
           "gpu_launches": int(launches), "clocks": clocks}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_autograd(args, local_rank, emit=True):
    """The 301 x 901, 20-shot gradient through the torch.autograd.Function
    (the differentiable-solver path): loss = 1/2 |d - d_obs|^2 of the
    modelled data, backward() for dJ/dv; end to end with the model and
    wavelets from pinned host memory and the gradient copied back."""
    import torch

    from paper_2604_14189_gb300 import autograd, sweep
    w = inputs.workload_marmousi(nshot=20, nt=3000)
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nshot, nt, nrec = 20, 3000, w["rec"].shape[1]
    p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                      nshot=nshot, nrec=nrec, f_ref=w["f0"])
    wav_h = torch.tensor(np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot),
                         dtype=torch.float32).pin_memory()
    v_h = torch.tensor(w["model"], dtype=torch.float32).pin_memory()
    src = torch.tensor(w["src"], device=dev)
    rec = torch.tensor(w["rec"], device=dev)
    d_obs = sweep.sweep_forward(p, torch.tensor(w["v_true"], dtype=torch.float32, device=dev),
                                wav_h.to(dev), src, rec)
    g_h = torch.empty((w["nz"], w["nx"]), dtype=torch.float32).pin_memory()

    def once():
        v = v_h.to(dev, non_blocking=True).requires_grad_(True)
        wav = wav_h.to(dev, non_blocking=True)
        d = autograd.acoustic_modelling(v, wav, p, src, rec)
        loss = 0.5 * ((d - d_obs).double() ** 2).sum()
        loss.backward()
        g_h.copy_(v.grad, non_blocking=True)
        return loss

    for _ in range(max(args.warmup, 1)):
        once()
    torch.cuda.synchronize()
    l0 = sweep.kernel_launches()
    t0 = time.perf_counter()
    runs = max(args.steps, 1)
    for _ in range(runs):
        loss = once()
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / runs
    c = counts(w["nz"], w["nx"], w["pml"])
    val = c["N_pad"] * nt * nshot / sec / 1e9
    out = {"metric": "Gpts/s fwd+adj (autograd.Function)", "value": val, "unit": "Gpts/s",
           "ms_per_step": sec * 1e3, "higher_is_better": True,
           "config": {"workload": "acoustic gradient 301x901 + 40 CPML, nt 3000, 20 shots, "
                                  "through AcousticModelling (forward, then backward = "
                                  "sweep_gradient with the data-space gradient as residual)",
                      "loss": float(loss.detach())},
           "e2e": {"value": val, "unit": "Gpts/s",
                   "h2d_bytes_per_step": (v_h.numel() + wav_h.numel()) * 4,
                   "d2h_bytes_per_step": g_h.numel() * 4},
           "gpu_launches": int(sweep.kernel_launches() - l0)}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def run_one_launch(args, local_rank, emit=True, deterministic=False):
    """The 301 x 901, 20-shot gradient through the time-loop kernels
    (SWEEP_F_ONE_LAUNCH: one cooperative launch per direction, grid barriers
    between each step's stencil and CPML phases) instead of two launches per
    step, or (deterministic=True) through the per-step kernels in their
    bitwise-reproducible mode (SWEEP_F_DETERMINISTIC); inputs resident on the
    device, one call per step."""
    import torch

    from paper_2604_14189_gb300 import sweep
    w = inputs.workload_marmousi(nshot=20, nt=args.nt)
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    nshot, nt, nrec = 20, args.nt, w["rec"].shape[1]
    flag = sweep.F_DETERMINISTIC if deterministic else sweep.F_ONE_LAUNCH
    p = sweep.problem(nz=w["nz"], nx=w["nx"], pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=nt,
                      nshot=nshot, nrec=nrec, f_ref=w["f0"], flags=flag)
    wav = torch.tensor(np.stack([inputs.ricker(w["f0"], w["dt"], nt)] * nshot),
                       dtype=torch.float32, device=dev)
    v = torch.tensor(w["model"], dtype=torch.float32, device=dev)
    src, rec = torch.tensor(w["src"], device=dev), torch.tensor(w["rec"], device=dev)
    d_obs = sweep.sweep_forward(p, torch.tensor(w["v_true"], dtype=torch.float32, device=dev),
                                wav, src, rec)
    ws = sweep.alloc_workspace(p, sweep.MODE_GRADIENT, dev)
    g = torch.empty_like(v)
    J = torch.empty((), dtype=torch.float64, device=dev)
    for _ in range(max(args.warmup, 1)):
        sweep.sweep_gradient(p, v, wav, src, rec, d_obs, grad=g, misfit=J, ws=ws)
    torch.cuda.synchronize()
    l0 = sweep.kernel_launches()
    t0 = time.perf_counter()
    runs = max(args.steps, 1)
    for _ in range(runs):
        sweep.sweep_gradient(p, v, wav, src, rec, d_obs, grad=g, misfit=J, ws=ws, sync=False)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / runs
    if sweep.status(ws) != sweep.OK:
        raise RuntimeError(f"one-launch gradient: status {sweep.status(ws)}")
    c = counts(w["nz"], w["nx"], w["pml"])
    val = c["N_pad"] * nt * nshot / sec / 1e9
    what = ("SWEEP_F_DETERMINISTIC (one writer per cell and phase)" if deterministic else
            "SWEEP_F_ONE_LAUNCH (one cooperative launch per direction)")
    out = {"metric": "Gpts/s fwd+adj (%s)" % ("deterministic mode" if deterministic
                                               else "time-loop kernels"),
           "value": val, "unit": "Gpts/s", "ms_per_step": sec * 1e3, "higher_is_better": True,
           "config": {"workload": f"acoustic gradient 301x901 + 40 CPML, nt {nt}, 20 shots, "
                                  + what},
           "gpu_launches": int(sweep.kernel_launches() - l0) // runs}
    if emit:
        print(json.dumps(out), flush=True)
    return out


def compact(out):
    keep = ("metric", "value", "unit", "ms_per_step", "higher_is_better", "roofline",
            "path_roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks")
    r = {k: out[k] for k in keep if k in out}
    cfg = out.get("config", {})
    r["workload"] = cfg.get("workload")
    for k in ("model_error_initial", "model_error_final", "gradients", "line_search_forwards",
              "streams", "padded_cell_steps", "loss"):
        if k in cfg:
            r[k] = cfg[k]
    return r


def run_extras(args, local_rank):
    """The other configurations of the solver, one short run each, attached
    to the headline line: the 200 x 200 single-shot forward, the 20-shot
    gradient through autograd and through the time-loop kernels, the 64-shot
    elastic forward, the 8-shot elastic gradient, the 256-model heterogeneous
    batch and the plain FWI."""
    base = dict(vars(args))
    out = {}
    runs = (
        ("acoustic_forward_200x200", dict(steps=5, warmup=3),
         lambda a: run_forward200(a, local_rank, emit=False)),
        ("acoustic_gradient_autograd_301x901", dict(steps=1, warmup=1),
         lambda a: run_autograd(a, local_rank, emit=False)),
        ("elastic_forward_500x1500_64shots", dict(steps=1, warmup=1, nt=3000,
                                                  workload="elastic-forward"),
         lambda a: run_elastic(a, 0, 1, local_rank, emit=False)),
        ("elastic_gradient_500x1500_8shots", dict(steps=2, warmup=1, nt=3000,
                                                  workload="elastic-gradient"),
         lambda a: run_elastic(a, 0, 1, local_rank, emit=False)),
        ("acoustic_gradient_one_launch_301x901", dict(steps=1, warmup=1),
         lambda a: run_one_launch(a, local_rank, emit=False)),
        ("acoustic_gradient_deterministic_301x901", dict(steps=2, warmup=1),
         lambda a: run_one_launch(a, local_rank, emit=False, deterministic=True)),
        ("batch_256_models", dict(steps=1, warmup=1),
         lambda a: run_batch(a, local_rank, emit=False)),
        ("fwi_plain_256x256", dict(steps=1, warmup=1),
         lambda a: run_fwi(a, local_rank, emit=False)),
    )
    for name, over, fn in runs:
        a = argparse.Namespace(**dict(base, **over))
        try:
            out[name] = compact(fn(a))
        except Exception as e:  # one failing extra must not hide the headline
            out[name] = {"error": repr(e)[:400]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["sweep", "reference"], default="sweep")
    ap.add_argument("--nt", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line only, without the other configurations' runs")
    ap.add_argument("--no-graph", action="store_true",
                    help="time direct sweep_gradient calls instead of a graph replay")
    ap.add_argument("--workload", default="acoustic-gradient",
                    choices=["acoustic-gradient", "elastic-forward", "elastic-gradient", "fwi",
                             "batch", "fwi-learned", "unet-conv", "unet-train",
                             "acoustic-gradient-one-launch",
                             "acoustic-gradient-deterministic"],
                    help="acoustic-gradient is the headline; the elastic workloads are "
                         "measured on request")
    ap.add_argument("--pairs", type=int, default=2000,
                    help="fwi-learned: solver-generated training pairs")
    ap.add_argument("--epochs", type=int, default=20, help="fwi-learned: training epochs")
    ap.add_argument("--heldout", type=int, default=50, help="fwi-learned: held-out models")
    ap.add_argument("--conv", default="8,64,64,256,128",
                    help="unet-conv: B,H,W,cin,cout of the timed convolution")
    ap.add_argument("--cos-min", type=float, default=0.0,
                    help="fwi-learned: smallest cosine with the plain direction at which the "
                         "learned direction is tried")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    # one survey of 20 shots per GPU; each rank models its own block of it
    # (weak scaling: 20 shots per GPU whatever the GPU count)
    from paper_2604_14189_gb300 import shots as _shots
    w = inputs.workload_marmousi(nt=args.nt, total_shots=20 * world,
                                 shots=_shots.shard(20 * world, rank, world))
    if args.impl == "reference":
        run_reference(args, w, rank)
        return
    if args.workload != "acoustic-gradient":
        if world > 1 and rank != 0:
            return  # one GPU per box: these workloads run as rank 0 only
        if args.workload == "fwi":
            run_fwi(args, local_rank)
        elif args.workload == "batch":
            run_batch(args, local_rank)
        elif args.workload == "fwi-learned":
            run_fwi_learned(args, local_rank)
        elif args.workload in ("unet-conv", "unet-train"):
            run_unet(args, local_rank)
        elif args.workload == "acoustic-gradient-one-launch":
            run_one_launch(args, local_rank)
        elif args.workload == "acoustic-gradient-deterministic":
            run_one_launch(args, local_rank, deterministic=True)
        else:
            run_elastic(args, rank, 1, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_sweep(args, w, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
