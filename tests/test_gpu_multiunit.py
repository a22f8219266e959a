"""Oracle parity of the acoustic kernels on their multi-unit paths.

The stencil kernels are persistent: one CTA per SM takes (tile, shot) units
round-robin through a 4-stage (forward) or 2-stage (backward) TMA pipeline
(32-row tiles; 7 and 3 stages with the 16-row tiles of SWEEP_F_ROWS16).
Small parity cases give every CTA at most one unit, so the stage reuse, the
mbarrier phase flips and the descriptor tables only run when there are many
more units than SMs.  These cases compare the CUDA path with the FP64 oracle
exactly there:

* the benchmark's grid (301 x 901 + 40, 381 x 981 padded, 96 units per
  shot) with 5 shots, both edge shots included (480 units, >= 3 backward
  units per CTA): gradient of the L2 misfit;
* the benchmark's launch itself (20 shots, 1920 units, ~12.6 per CTA) in
  residual mode with a residual on 3 of the shots, so that the oracle needs
  only those 3 (the other shots' adjoint fields are zero);
* 129 x 133 + 11 with 64 shots (640 units, ~4.2 per CTA: every forward and
  backward stage is reused);
* 150 shots, more than the shared-memory shot table holds (128): the
  kernels read the source cell and wavelet sample from global memory;
* 48 000 one-tile shots: > 256 units per CTA, beyond the per-CTA table of
  unit descriptors, so later units are described into the stage ring;
* the 5-shot full-size gradient, the 64-shot and the 48 000-shot cases again
  in 16-row tiles.

Beside the global relative L2 (<= 1e-4 seismograms, <= 1e-3 gradients) each
case checks every trace on its own (<= 1e-3), and the gradient in the 4-cell
band inside the interior edge (where the forward ring is restored) and in
the 9 x 9 neighbourhood of every source (<= 1e-3 each), so that an error
confined to a few tiles, one trace or one region cannot hide under the
global norm.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_14189_gb300 import inputs
from parity_util import assert_gradient, rel, worst_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import sweep
    return sweep


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def cuda(x, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)


# ----------------------------------------------------------- full-size grid
NT_FULL = 600  # the oracle's gradient at 381 x 981 takes ~30 s for 5 shots
PICK5 = [0, 5, 10, 14, 19]  # x = 0 ... 900: both edge shots


@pytest.fixture(scope="module")
def full(sw):
    w = inputs.workload_marmousi(nshot=20, nt=NT_FULL)
    nrec = w["rec"].shape[1]
    wav = np.stack([inputs.ricker(w["f0"], w["dt"], NT_FULL)] * 20).astype(np.float32)
    q5 = oracle.make_problem(0, w["nz"], w["nx"], w["pml"], np.float32(w["dx"]),
                             np.float32(w["dt"]), NT_FULL, len(PICK5), nrec,
                             np.float32(w["f0"]))
    oracle.set_threads(len(PICK5))
    d_obs5 = oracle.acoustic_forward(q5, f32(w["v_true"]), wav[PICK5].astype(np.float64),
                                     w["src"][PICK5], w["rec"][PICK5])
    return w, wav, d_obs5, {}


@pytest.mark.parametrize("rows16", [False, True])
def test_fullsize_five_shot_gradient_matches_oracle(sw, full, rows16):
    """Both stencil tile heights: 32 rows (12 x 8 = 96 units per shot) and
    16 rows (24 x 8 = 192 units per shot, 7 forward and 3 backward stages)."""
    w, wav, d_obs5, memo = full
    nz, nx, nrec = w["nz"], w["nx"], w["rec"].shape[1]
    assert list(w["src"][[PICK5[0], PICK5[-1]], 1]) == [0, 900]
    p = sw.problem(nz=nz, nx=nx, pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=NT_FULL, nshot=5,
                   nrec=nrec, f_ref=w["f0"], flags=sw.F_ROWS16 if rows16 else 0)
    q = oracle.make_problem(0, nz, nx, w["pml"], np.float32(w["dx"]), np.float32(w["dt"]),
                            NT_FULL, 5, nrec, np.float32(w["f0"]))
    src, rec = w["src"][PICK5], w["rec"][PICK5]
    g, J, _ = sw.sweep_gradient(p, cuda(w["model"]), cuda(wav[PICK5]), cuda(src, torch.int32),
                                cuda(rec, torch.int32), cuda(d_obs5[:, None]))
    if "g5" not in memo:  # the oracle's gradient serves both tile heights
        oracle.set_threads(5)
        memo["g5"] = oracle.acoustic_gradient(q, f32(w["model"]), f32(wav[PICK5]), src, rec,
                                              f32(d_obs5))
    gref, Jref = memo["g5"]
    assert abs(J.item() - Jref) <= 1e-4 * Jref, (J.item(), Jref)
    assert_gradient(g.cpu().numpy(), gref, src)


def test_fullsize_twenty_shot_launch_matches_oracle(sw, full):
    """The benchmark's 20-shot launch (1920 units per stencil launch),
    residual mode: shots 0, 10, 19 carry a residual, the others none."""
    w, wav, d_obs5, _ = full
    nz, nx, nrec = w["nz"], w["nx"], w["rec"].shape[1]
    carry = [0, 10, 19]
    r = np.zeros((20, 1, nrec, NT_FULL), dtype=np.float32)
    for s in carry:
        r[s, 0] = d_obs5[PICK5.index(s)]
    p = sw.problem(nz=nz, nx=nx, pml=w["pml"], dx=w["dx"], dt=w["dt"], nt=NT_FULL, nshot=20,
                   nrec=nrec, f_ref=w["f0"], flags=sw.F_RESIDUAL_IN)
    g, J, _ = sw.sweep_gradient(p, cuda(w["model"]), cuda(wav), cuda(w["src"], torch.int32),
                                cuda(w["rec"], torch.int32), cuda(r))
    q = oracle.make_problem(0, nz, nx, w["pml"], np.float32(w["dx"]), np.float32(w["dt"]),
                            NT_FULL, len(carry), nrec, np.float32(w["f0"]), sw.F_RESIDUAL_IN)
    oracle.set_threads(len(carry))
    gref, Jref = oracle.acoustic_gradient(q, f32(w["model"]), f32(wav[carry]), w["src"][carry],
                                          w["rec"][carry], f32(r[carry, 0]))
    assert abs(J.item() - Jref) <= 1e-6 * Jref
    assert_gradient(g.cpu().numpy(), gref, w["src"][carry])


# ------------------------------------------------------ many units per CTA
def layered_case(nz, nx, nshot, nrec, seed):
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None]
    v = 1800.0 + 1000.0 * z / max(nz - 1, 1) + 120.0 * rng.standard_normal((nz, nx))
    v = np.clip(v, 1500.0, 3200.0)
    src = np.stack([rng.integers(0, nz, nshot), rng.integers(0, nx, nshot)], -1)
    rec = np.stack([rng.integers(0, nz, (nshot, nrec)), rng.integers(0, nx, (nshot, nrec))], -1)
    return v, src.astype(np.int32), rec.astype(np.int32)


def run_case(sw, nz, nx, pml, nt, nshot, nrec, seed, f0=15.0, threads=None, flags=0):
    v, src, rec = layered_case(nz, nx, nshot, nrec, seed)
    rng = np.random.default_rng(seed + 1)
    wav = np.stack([inputs.ricker(f0 * (1 + 0.2 * rng.random()), 1e-3, nt)
                    for _ in range(nshot)]).astype(np.float32)
    v_true = v * (1 + 0.03 * rng.standard_normal(v.shape))
    p = sw.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=nshot, nrec=nrec,
                   f_ref=f0, flags=flags)
    q = oracle.make_problem(0, nz, nx, pml, np.float32(10.0), np.float32(1e-3), nt, nshot, nrec,
                            np.float32(f0))
    oracle.set_threads(threads)
    ref = oracle.acoustic_forward(q, f32(v), f32(wav), src, rec)
    d_obs = oracle.acoustic_forward(q, f32(v_true), f32(wav), src, rec)
    tv, tw = cuda(v), cuda(wav)
    ts, tr = cuda(src, torch.int32), cuda(rec, torch.int32)
    d = sw.sweep_forward(p, tv, tw, ts, tr).cpu().numpy()[:, 0]
    assert rel(d, ref) <= 1e-4, rel(d, ref)
    assert worst_trace(d, ref) <= 1e-3, worst_trace(d, ref)
    g, J, _ = sw.sweep_gradient(p, tv, tw, ts, tr, cuda(d_obs[:, None]))
    gref, Jref = oracle.acoustic_gradient(q, f32(v), f32(wav), src, rec, f32(d_obs))
    nd, nr = np.linalg.norm(ref), np.linalg.norm(ref - f32(d_obs))
    assert abs(J.item() - Jref) <= 1e-4 * nd * nr + 0.5e-8 * nd ** 2
    assert_gradient(g.cpu().numpy(), gref, src)


def test_stage_reuse_64_shots(sw):
    """129 x 133 + 11: 5 x 2 tiles per shot, 640 units, every forward (4)
    and backward (2) pipeline stage used several times by each CTA."""
    run_case(sw, 129, 133, 11, 220, 64, 9, seed=101)


def test_stage_reuse_64_shots_16_row_tiles(sw):
    """The same grid in 16-row tiles: 10 x 2 tiles per shot, 1280 units,
    ~8.4 per CTA through 7 forward and 3 backward stages."""
    run_case(sw, 129, 133, 11, 220, 64, 9, seed=104, flags=sw.F_ROWS16)


def test_more_shots_than_the_shot_table(sw):
    """150 shots > 128: source cells and wavelet samples come from global
    memory in every unit descriptor."""
    run_case(sw, 37, 45, 6, 160, 150, 5, seed=102)


def test_more_units_than_the_descriptor_table(sw):
    """48 000 one-tile shots (18 x 20 padded): ~316 units per CTA on 152
    SMs, past the 256 descriptors a CTA computes in its prologue."""
    nshot = 48000
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert nshot / sms > 256
    run_case(sw, 10, 12, 4, 40, nshot, 2, seed=103)


def test_more_units_than_the_descriptor_table_16_row_tiles(sw):
    """16-row tiles of the same 18 x 20 padded grid: 2 tiles per shot,
    ~632 units per CTA, most of them described into the stage ring."""
    run_case(sw, 10, 12, 4, 40, 48000, 2, seed=105, flags=sw.F_ROWS16)
