"""Heterogeneous batches: the LPT schedule (CPU) and batch runs equal to
one-by-one runs (GPU)."""
import itertools
import json

import numpy as np
import pytest
import torch

from paper_2604_14189_gb300 import batch


def _optimal_makespan(costs, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        load = [0] * m
        for c, k in zip(costs, assign):
            load[k] += c
        best = min(best, max(load))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_schedule_covers_every_job_once_within_lpt_bound(seed):
    rng = np.random.default_rng(seed)
    costs = [int(c) for c in rng.integers(1, 100, 7)]
    m = int(rng.integers(1, 4))
    q = batch.schedule(costs, m)
    assert sorted(j for s in q for j in s) == list(range(len(costs)))
    makespan = max(sum(costs[j] for j in s) for s in q)
    opt = _optimal_makespan(costs, m)
    assert makespan <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9


def test_schedule_deals_longest_first():
    q = batch.schedule([5, 9, 1, 7], 2)
    # 9 -> s0, 7 -> s1, 5 -> s1 (7 < 9), 1 -> s0 (9 < 12)
    assert q == [[1, 2], [3, 0]]
    with pytest.raises(ValueError):
        batch.schedule([1], 0)


def test_cohorts_group_similar_record_lengths():
    from types import SimpleNamespace as NS
    rng = np.random.default_rng(3)
    nts = rng.integers(100, 3000, 37)
    items = [NS(problem=NS(nt=int(t), nz=10, nx=10, pml=2, nshot=1)) for t in nts]
    groups = batch.cohorts(items, size=16)
    assert [len(g) for g in groups] == [16, 16, 5]
    assert sorted(i for g in groups for i in g) == list(range(37))
    flat = [int(nts[i]) for g in groups for i in g]
    assert flat == sorted(flat, reverse=True)


def test_tune_cache_skips_timing_for_a_known_batch(tmp_path, monkeypatch):
    """The stream-count autotuner stores its choice per (GPU model, mode,
    candidates, problem sizes) and takes it from the cache next time without
    running anything; another batch or GPU model is timed afresh."""
    from types import SimpleNamespace as NS

    from paper_2604_14189_gb300 import sweep
    ran = []
    monkeypatch.setattr(batch, "run", lambda items, mode, n, device, fused: ran.append(n))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    gpu = ["GB300"]
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: gpu[0])
    items = [NS(problem=sweep.problem(nz=40 + i, nx=50, pml=10, dx=10.0, dt=1e-3, nt=100,
                                      nshot=1, nrec=5)) for i in range(3)]
    path = str(tmp_path / "tune.json")
    best, times = batch.autotune_streams(items, candidates=(1, 2, 3), cache=path)
    assert ran == [1, 2, 3] and best in (1, 2, 3) and set(times) == {1, 2, 3}
    ran.clear()
    assert batch.autotune_streams(items, candidates=(1, 2, 3), cache=path) == (best, times)
    assert ran == []  # taken from the cache
    batch.autotune_streams(items[:2], candidates=(1, 2, 3), cache=path)
    assert ran == [1, 2, 3]  # other problem sizes
    ran.clear()
    gpu[0] = "another GPU"
    batch.autotune_streams(items, candidates=(1, 2, 3), cache=path)
    assert ran == [1, 2, 3]
    ran.clear()
    monkeypatch.setenv("SWEEP_TUNE_CACHE", path)  # the default cache location
    batch.autotune_streams(items, candidates=(1, 2, 3))
    assert ran == []
    assert len(json.load(open(path))) == 3


def test_tile_tuner_sets_flags_by_size_and_caches(tmp_path, monkeypatch):
    """The tile-height tuner times each threshold with the items' flags set
    by it (16-row tiles below the threshold only, acoustic only, other flag
    bits kept), leaves the fastest setting on the items and takes it from
    the cache next time without running anything."""
    from types import SimpleNamespace as NS

    from paper_2604_14189_gb300 import sweep
    seen = []

    def fake_run(items, mode, n, device, fused):
        seen.append([bool(it.problem.flags & sweep.F_ROWS16) for it in items])
    monkeypatch.setattr(batch, "run", fake_run)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GB300")
    clock = iter(range(1000))
    monkeypatch.setattr(batch.time, "perf_counter", lambda: float(next(clock)) ** 2)
    kw = dict(dx=10.0, dt=1e-3, nt=100, nrec=5)
    # 32-row units: 1 x 1 x 1 = 1, 4 x 2 x 2 = 16, 10 x 3 x 4 = 120; elastic 1
    items = [NS(problem=sweep.problem(nz=20, nx=20, pml=4, nshot=1, **kw)),
             NS(problem=sweep.problem(nz=100, nx=200, pml=10, nshot=2,
                                      flags=sweep.F_PADDED_MODEL, **kw)),
             NS(problem=sweep.problem(nz=300, nx=300, pml=10, nshot=4, **kw)),
             NS(problem=sweep.problem(sweep.ELASTIC, nz=20, nx=20, pml=4, nshot=1, **kw))]
    assert [batch.stencil_units(it.problem) for it in items] == [1, 16, 120, 1]
    path = str(tmp_path / "tune.json")
    best, times = batch.autotune_tiles(items, thresholds=(0, 2, 100, 1000), cache=path)
    assert seen == [[False, False, False, False], [True, False, False, False],
                    [True, True, False, False], [True, True, True, False]]
    # the fake clock makes later candidates slower: threshold 0 wins
    assert best == 0 and sorted(times) == [0, 2, 100, 1000]
    assert not any(it.problem.flags & sweep.F_ROWS16 for it in items)
    assert items[1].problem.flags == sweep.F_PADDED_MODEL  # other bits kept
    seen.clear()
    batch.set_tiles(items, 1000)
    assert batch.autotune_tiles(items, thresholds=(0, 2, 100, 1000), cache=path) == (best, times)
    assert seen == []  # taken from the cache, and applied
    assert not any(it.problem.flags & sweep.F_ROWS16 for it in items)
    batch.autotune_tiles(items, thresholds=(0, 2, 100, 1000), streams=3, cache=path)
    assert len(seen) == 4  # another stream count is another key


def test_output_shapes_follow_the_physics():
    """Outputs allocated by run() have the sizes the C ABI writes: an
    elastic problem has three gradients and two data components."""
    from paper_2604_14189_gb300 import sweep
    kw = dict(nz=7, nx=9, pml=3, dx=10.0, dt=1e-3, nt=11, nshot=2, nrec=5)
    assert batch.out_shapes(sweep.problem(sweep.ACOUSTIC, **kw)) == ((7, 9), (2, 1, 5, 11))
    assert batch.out_shapes(sweep.problem(sweep.ELASTIC, **kw)) == ((3, 7, 9), (2, 2, 5, 11))


@pytest.mark.gpu
@pytest.mark.parametrize("count,fused", [(6, True), (6, False), (21, True)])
def test_batch_matches_individual_runs(count, fused):
    """Shared-launch cohorts (21 problems: a full cohort of 16 and one of 5)
    and the one-call-per-problem path give the problems' own gradients."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import inputs, sweep

    rng = np.random.default_rng(7)
    items, refs = [], []
    for k in range(count):
        nz, nx = int(rng.integers(40, 90)), int(rng.integers(40, 120))
        pml, nt, ns = int(rng.integers(8, 20)), int(rng.integers(150, 400)), int(rng.integers(1, 4))
        z = np.arange(nz)[:, None] + np.zeros((1, nx))
        v = np.where(z < nz // 3, 1800.0, np.where(z < 2 * nz // 3, 2300.0, 2900.0))
        sx = np.round(np.linspace(1, nx - 2, ns)).astype(np.int32)
        src = np.stack([np.full(ns, 2), sx], -1).astype(np.int32)
        rec = inputs.surface_line(ns, 2, np.arange(0, nx, 2))
        p = sweep.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=ns,
                          nrec=rec.shape[1], f_ref=10.0)
        dev = "cuda"
        w = torch.tensor(np.stack([inputs.ricker(10.0, 1e-3, nt)] * ns), dtype=torch.float32,
                         device=dev)
        vt = torch.tensor(v, dtype=torch.float32, device=dev)
        st, rt = torch.tensor(src, device=dev), torch.tensor(rec, device=dev)
        d_obs = sweep.sweep_forward(p, vt * 1.02, w, st, rt)
        items.append(batch.Item(p, vt, w, st, rt, d_obs=d_obs))
        g, J, _ = sweep.sweep_gradient(p, vt, w, st, rt, d_obs)
        refs.append((g.clone(), float(J)))
    codes = batch.run(items, streams=3, fused=fused)
    assert codes == [0] * len(items)
    for it, (g, J) in zip(items, refs):
        assert torch.linalg.norm(it.grad - g) <= 1e-4 * torch.linalg.norm(g)
        # corner cells receive their two CPML additions in either order, and a
        # small residual amplifies the run-to-run rounding differences
        assert abs(float(it.misfit) - J) <= 1e-4 * J


@pytest.mark.gpu
def test_deterministic_batch_equals_individual_runs_bitwise():
    """In deterministic mode the shared-launch cohort (9 uneven problems,
    some in 16-row tiles) gives each problem's own gradient and misfit bit
    for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import inputs, sweep

    rng = np.random.default_rng(19)
    items, refs = [], []
    dev = "cuda"
    for k in range(9):
        nz, nx = int(rng.integers(40, 90)), int(rng.integers(40, 120))
        pml, nt, ns = int(rng.integers(8, 20)), int(rng.integers(150, 300)), int(rng.integers(1, 4))
        v = np.clip(1800.0 + 900.0 * np.arange(nz)[:, None] / nz +
                    80.0 * rng.standard_normal((nz, nx)), 1500.0, 3000.0)
        src = np.stack([np.full(ns, 2), rng.integers(0, nx, ns)], -1).astype(np.int32)
        rec = inputs.surface_line(ns, 2, np.arange(0, nx, 2))
        flags = sweep.F_DETERMINISTIC | (sweep.F_ROWS16 if k % 3 == 0 else 0)
        p = sweep.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=ns,
                          nrec=rec.shape[1], f_ref=10.0, flags=flags)
        w = torch.tensor(np.stack([inputs.ricker(10.0, 1e-3, nt)] * ns), dtype=torch.float32,
                         device=dev)
        vt = torch.tensor(v, dtype=torch.float32, device=dev)
        st, rt = torch.tensor(src, device=dev), torch.tensor(rec, device=dev)
        d_obs = sweep.sweep_forward(p, vt * 1.02, w, st, rt)
        items.append(batch.Item(p, vt, w, st, rt, d_obs=d_obs))
        g, J, _ = sweep.sweep_gradient(p, vt, w, st, rt, d_obs)
        refs.append((g.clone(), float(J)))
    assert batch.run(items, streams=2) == [0] * len(items)
    for it, (g, J) in zip(items, refs):
        assert torch.equal(it.grad, g) and float(it.misfit) == J


@pytest.mark.gpu
def test_forward_batch_matches_individual_runs():
    """Forward modelling of 19 uneven problems as cohorts sharing launches
    (a cohort of 16 and one of 3) equals each problem's own sweep_forward
    to rounding (1e-5 of the largest sample)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import inputs, sweep

    rng = np.random.default_rng(11)
    items, refs = [], []
    dev = "cuda"
    for k in range(19):
        nz, nx = int(rng.integers(30, 100)), int(rng.integers(30, 140))
        pml, nt, ns = int(rng.integers(0, 16)), int(rng.integers(60, 300)), int(rng.integers(1, 4))
        v = 1800.0 + 600.0 * rng.random((nz, nx))
        src = np.stack([rng.integers(0, nz, ns), rng.integers(0, nx, ns)], -1).astype(np.int32)
        rec = np.stack([rng.integers(0, nz, (ns, 5)), rng.integers(0, nx, (ns, 5))],
                       -1).astype(np.int32)
        p = sweep.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=ns, nrec=5,
                          f_ref=10.0)
        w = torch.tensor(np.stack([inputs.ricker(12.0, 1e-3, nt)] * ns), dtype=torch.float32,
                         device=dev)
        it = batch.Item(p, torch.tensor(v, dtype=torch.float32, device=dev), w,
                        torch.tensor(src, device=dev), torch.tensor(rec, device=dev))
        items.append(it)
        refs.append(sweep.sweep_forward(p, it.model, it.wavelet, it.src, it.rec).clone())
    codes = batch.run(items, mode=sweep.MODE_FORWARD, streams=2)
    assert codes == [0] * len(items)
    for it, ref in zip(items, refs):
        scale = float(ref.abs().max())
        assert scale > 0 and float((it.data - ref).abs().max()) <= 1e-5 * scale


@pytest.mark.gpu
def test_batch_cohort_matches_oracle():
    """One shared-launch cohort of 16 uneven problems (the persistent CTAs
    split per problem, the CPML blocks laid end to end): 4 of its problems'
    gradients and misfits against the FP64 oracle (relative L2 <= 1e-3 for
    the gradient, and the misfit within the bound the seismogram tolerance
    gives), not only against the library's one-problem calls."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2604_14189_gb300 import inputs, sweep

    rng = np.random.default_rng(17)
    items, cases = [], []
    dev = "cuda"
    for k in range(16):
        nz, nx = int(rng.integers(30, 80)), int(rng.integers(30, 110))
        pml, nt, ns = int(rng.integers(6, 18)), int(rng.integers(120, 260)), int(rng.integers(1, 4))
        z = np.arange(nz)[:, None]
        v = np.clip(1800.0 + 900.0 * z / nz + 100.0 * rng.standard_normal((nz, nx)), 1500, 3000)
        vt = v * (1 + 0.03 * rng.standard_normal(v.shape))
        src = np.stack([np.full(ns, 2), rng.integers(0, nx, ns)], -1).astype(np.int32)
        rec = inputs.surface_line(ns, 1, np.arange(0, nx, 3))
        wav = np.stack([inputs.ricker(12.0, 1e-3, nt)] * ns).astype(np.float32)
        p = sweep.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=ns,
                          nrec=rec.shape[1], f_ref=12.0)
        q = oracle.make_problem(0, nz, nx, pml, np.float32(10.0), np.float32(1e-3), nt, ns,
                                rec.shape[1], np.float32(12.0))
        v32 = np.float32(v).astype(np.float64)
        w64 = wav.astype(np.float64)
        d_obs = oracle.acoustic_forward(q, np.float32(vt).astype(np.float64), w64, src, rec)
        items.append(batch.Item(p, torch.tensor(v, dtype=torch.float32, device=dev),
                                torch.tensor(wav, device=dev), torch.tensor(src, device=dev),
                                torch.tensor(rec, device=dev),
                                d_obs=torch.tensor(d_obs[:, None], dtype=torch.float32,
                                                   device=dev)))
        cases.append((q, v32, w64, src, rec, np.float32(d_obs).astype(np.float64)))
    assert batch.run(items, streams=1, fused=True) == [0] * 16
    for k in (0, 5, 10, 15):
        q, v32, w64, src, rec, d_obs = cases[k]
        gref, Jref = oracle.acoustic_gradient(q, v32, w64, src, rec, d_obs)
        d_ref = oracle.acoustic_forward(q, v32, w64, src, rec)
        nd, nr = np.linalg.norm(d_ref), np.linalg.norm(d_ref - d_obs)
        g = items[k].grad.double().cpu().numpy()
        err = np.linalg.norm(g - gref) / np.linalg.norm(gref)
        assert err <= 1e-3, (k, err)
        assert abs(float(items[k].misfit) - Jref) <= 1e-4 * nd * nr + 0.5e-8 * nd ** 2, k
