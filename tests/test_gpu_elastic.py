"""Parity of the CUDA elastic (velocity-stress, staggered) forward with the
FP64 oracle, through the C ABI.  Tolerance: seismograms relative L2 <= 1e-4."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_14189_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import sweep
    return sweep


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def run_both(sw, model, nz, nx, pml, dx, dt, nt, f0, src, rec, flags=0):
    nshot, nrec = src.shape[0], rec.shape[1]
    w = np.stack([inputs.ricker(f0 * (1 + 0.05 * k), dt, nt) for k in range(nshot)])
    p = sw.problem(sw.ELASTIC, nz=nz, nx=nx, pml=pml, dx=dx, dt=dt, nt=nt, nshot=nshot,
                   nrec=nrec, f_ref=f0, flags=flags)
    q = oracle.make_problem(1, nz, nx, pml, np.float32(dx), np.float32(dt), nt, nshot, nrec,
                            np.float32(f0), flags)
    dev = "cuda"
    d = sw.sweep_forward(p, torch.tensor(model, dtype=torch.float32, device=dev),
                         torch.tensor(w, dtype=torch.float32, device=dev),
                         torch.tensor(src, dtype=torch.int32, device=dev),
                         torch.tensor(rec, dtype=torch.int32, device=dev)).cpu().numpy()
    ref = oracle.elastic_forward(q, f32(model), f32(w), src, rec)
    return d, ref


def random_model(nz, nx, seed):
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None]
    vp = 2000.0 + 1500.0 * z / nz + 100.0 * rng.standard_normal((nz, nx))
    vs = vp / rng.uniform(1.6, 2.0, (nz, nx))
    rho = 310.0 * vp ** 0.25
    return np.stack([vp, vs, rho])


@pytest.mark.parametrize("shape", [(37, 45, 6, 300, 2, 5), (70, 150, 20, 400, 3, 20),
                                   (9, 11, 4, 150, 1, 3)])
def test_elastic_forward_matches_oracle(sw, shape):
    nz, nx, pml, nt, nshot, nrec = shape
    rng = np.random.default_rng(sum(shape))
    m = random_model(nz, nx, sum(shape))
    src = np.stack([rng.integers(0, nz, nshot), rng.integers(0, nx, nshot)], -1)
    rec = np.stack([rng.integers(0, nz, (nshot, nrec)), rng.integers(0, nx, (nshot, nrec))], -1)
    d, ref = run_both(sw, m, nz, nx, pml, 5.0, 4e-4, nt, 25.0, src, rec)
    assert np.abs(ref).max() > 0
    assert rel(d, ref) <= 1e-4, rel(d, ref)


def layered_model(ex, nz, nx):
    """The three-layer model of tests/golden/layered_example.json (the
    paper's Sec. 3.6.1 example: a fluid over two solids) on an nz x nx
    grid, layers of equal thickness: [3][nz][nx]."""
    z = np.arange(nz)[:, None] * 3 // nz + np.zeros((1, nx), dtype=int)
    return np.stack([np.asarray(ex[k])[z] for k in ("vp_m_s", "vs_m_s", "rho_kg_m3")])


def test_elastic_three_layer_fluid_top(sw, golden):
    """Forward on the paper's three-layer example (no-shear top layer)."""
    ex = golden("layered_example.json")
    nz, nx = 90, 120
    src = np.array([[10, 60]])
    rec = inputs.surface_line(1, 5, np.arange(0, nx, 4))
    d, ref = run_both(sw, layered_model(ex, nz, nx), nz, nx, 20, 10.0, 1e-3, 500,
                      ex["ricker_peak_hz"], src, rec)
    assert rel(d, ref) <= 1e-4, rel(d, ref)


def test_elastic_padded_model_and_errors(sw):
    nz, nx, pml = 30, 40, 8
    m = random_model(nz, nx, 5)
    mp = inputs.pad_edge(m, pml)
    mp[2, :4] *= 1.2  # padding values are used
    src = np.array([[3, 7], [20, 30]])
    rec = np.array([[[0, 0], [10, 10]], [[29, 39], [5, 5]]])
    d, ref = run_both(sw, mp, nz, nx, pml, 5.0, 4e-4, 200, 25.0, src, rec,
                      flags=sw.F_PADDED_MODEL)
    assert rel(d, ref) <= 1e-4
    p = sw.problem(sw.ELASTIC, nz=nz, nx=nx, pml=pml, dx=5.0, dt=2e-3, nt=10, nshot=2, nrec=2)
    with pytest.raises(sw.SweepError) as e:  # 4000 m/s * 2 ms / 5 m > 0.606
        sw.sweep_forward(p, torch.tensor(m, dtype=torch.float32, device="cuda"),
                         torch.zeros((2, 10), device="cuda"),
                         torch.tensor(src, dtype=torch.int32, device="cuda"),
                         torch.tensor(rec, dtype=torch.int32, device="cuda"))
    assert e.value.code == sw.ECFL
    bad = m.copy()
    bad[1, 3, 3] = bad[0, 3, 3]  # vs = vp: negative lambda
    p2 = sw.problem(sw.ELASTIC, nz=nz, nx=nx, pml=pml, dx=5.0, dt=4e-4, nt=10, nshot=2, nrec=2)
    with pytest.raises(sw.SweepError) as e:
        sw.sweep_forward(p2, torch.tensor(bad, dtype=torch.float32, device="cuda"),
                         torch.zeros((2, 10), device="cuda"),
                         torch.tensor(src, dtype=torch.int32, device="cuda"),
                         torch.tensor(rec, dtype=torch.int32, device="cuda"))
    assert e.value.code == sw.EMODEL


def test_elastic_workload_grid_reduced_shots(sw):
    """The 500 x 1500 (dx 5 m, dt 0.5 ms, 15 Hz, 40-cell CPML) elastic grid
    with 2 of its 64 shots and 300 of its 4000 steps, 750 receivers."""
    wl = inputs.workload_elastic(nshot=2, nt=300)
    src = wl["src"][[0, 1]]
    src[1] = [2, 750]
    d, ref = run_both(sw, wl["model"], wl["nz"], wl["nx"], wl["pml"], wl["dx"], wl["dt"],
                      wl["nt"], wl["f0"], src, wl["rec"])
    assert rel(d, ref) <= 1e-4, rel(d, ref)


# ------------------------------------------------------------ adjoint (E5)
def _tensors(sw, model, w, src, rec):
    dev = "cuda"
    return (torch.tensor(model, dtype=torch.float32, device=dev),
            torch.tensor(w, dtype=torch.float32, device=dev),
            torch.tensor(src, dtype=torch.int32, device=dev),
            torch.tensor(rec, dtype=torch.int32, device=dev))


def _setup(seed, nz=37, nx=45, pml=8, nt=240, nshot=2, nrec=7):
    rng = np.random.default_rng(seed)
    m = random_model(nz, nx, seed)
    src = np.stack([rng.integers(2, nz - 2, nshot), rng.integers(2, nx - 2, nshot)], -1)
    rec = np.stack([rng.integers(0, nz, (nshot, nrec)), rng.integers(0, nx, (nshot, nrec))], -1)
    dt, dx, f0 = 4e-4, 5.0, 25.0
    w = np.stack([inputs.ricker(f0 * (1 + 0.05 * k), dt, nt) for k in range(nshot)]) * 1e6
    return m, src, rec, w, dict(nz=nz, nx=nx, pml=pml, dx=dx, dt=dt, nt=nt, nshot=nshot,
                                nrec=nrec, f0=f0), rng


def test_elastic_adjoint_matches_oracle(sw):
    m, src, rec, w, c, rng = _setup(11)
    p = sw.problem(sw.ELASTIC, nz=c["nz"], nx=c["nx"], pml=c["pml"], dx=c["dx"], dt=c["dt"],
                   nt=c["nt"], nshot=c["nshot"], nrec=c["nrec"], f_ref=c["f0"], v_pml=4000.0)
    q = oracle.make_problem(1, c["nz"], c["nx"], c["pml"], np.float32(c["dx"]),
                            np.float32(c["dt"]), c["nt"], c["nshot"], c["nrec"],
                            np.float32(c["f0"]), v_pml=4000.0)
    adj = rng.standard_normal((c["nshot"], 2, c["nrec"], c["nt"])).astype(np.float32)
    mt, wt, st, rt = _tensors(sw, m, w, src, rec)
    wg = sw.sweep_adjoint(p, mt, torch.tensor(adj, device="cuda"), st, rt).cpu().numpy()
    ref = oracle.elastic_adjoint(q, f32(m), adj.astype(np.float64), src, rec)
    assert rel(wg, ref) <= 1e-4, rel(wg, ref)


def test_elastic_dot_product_on_gpu(sw):
    """<F w, d> = <w, F^T d> with both sides from the CUDA path (FP64 sums)."""
    m, src, rec, w, c, rng = _setup(12)
    p = sw.problem(sw.ELASTIC, nz=c["nz"], nx=c["nx"], pml=c["pml"], dx=c["dx"], dt=c["dt"],
                   nt=c["nt"], nshot=c["nshot"], nrec=c["nrec"], f_ref=c["f0"])
    mt, wt, st, rt = _tensors(sw, m, w, src, rec)
    d = sw.sweep_forward(p, mt, wt, st, rt)
    db = torch.randn(d.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    wg = sw.sweep_adjoint(p, mt, db, st, rt)
    lhs = float(sw.sweep_dot(d.reshape(-1), db.reshape(-1)))
    rhs = float(sw.sweep_dot(wt.reshape(-1), wg.reshape(-1)))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("seed,nt", [(13, 240), (14, 97)])
def test_elastic_gradient_matches_oracle(sw, seed, nt):
    """(vp, vs, rho) gradient of the CUDA path (checkpointed replay, nt not a
    square: ragged last segment) against the FP64 reverse-mode oracle;
    relative L2 per parameter <= 1e-3, misfit within the trace tolerance."""
    m, src, rec, w, c, rng = _setup(seed, nt=nt)
    mt = m.copy()
    mt[0, 12:20, 15:25] *= 1.04
    mt[1, 20:28, 10:22] *= 0.95
    mt[2, 8:16, 25:35] *= 1.05
    p = sw.problem(sw.ELASTIC, nz=c["nz"], nx=c["nx"], pml=c["pml"], dx=c["dx"], dt=c["dt"],
                   nt=nt, nshot=c["nshot"], nrec=c["nrec"], f_ref=c["f0"], v_pml=4000.0)
    q = oracle.make_problem(1, c["nz"], c["nx"], c["pml"], np.float32(c["dx"]),
                            np.float32(c["dt"]), nt, c["nshot"], c["nrec"], np.float32(c["f0"]),
                            v_pml=4000.0)
    dobs = oracle.elastic_forward(q, f32(mt), f32(w), src, rec).astype(np.float32)
    mtt, wt, st, rt = _tensors(sw, m, w, src, rec)
    g, J, _ = sw.sweep_gradient(p, mtt, wt, st, rt, torch.tensor(dobs, device="cuda"))
    g = g.cpu().numpy()
    gref, Jref = oracle.elastic_gradient(q, f32(m), f32(w), src, rec, dobs.astype(np.float64))
    assert abs(float(J) - Jref) <= 2e-3 * Jref, (float(J), Jref)
    for k in range(3):
        assert np.abs(gref[k]).max() > 0
        assert rel(g[k], gref[k]) <= 1e-3, (k, rel(g[k], gref[k]))


def test_elastic_gradient_layered_fluid_top(sw, golden):
    """(vp, vs, rho) gradient on the paper's three-layer example, whose top
    layer has no shear modulus: the harmonic shear average and its chain rule
    must skip the fluid on both sides; relative L2 per parameter <= 1e-3."""
    ex = golden("layered_example.json")
    nz, nx, pml, dx, dt, nt, f0 = 48, 56, 8, 10.0, 1e-3, 400, ex["ricker_peak_hz"]
    m = layered_model(ex, nz, nx)   # fluid rows 0..15, solids 16..31, 32..47
    mt = m.copy()
    mt[0, 20:28, 20:34] *= 1.05   # middle layer
    mt[1, 22:30, 10:24] *= 0.95   # middle layer
    mt[2, 4:12, 30:44] *= 1.04    # fluid layer
    # sources in the middle layer (P and S in the solid, converted at the
    # fluid interface); receivers in the fluid and in the bottom layer, so
    # that the three gradients are of like size
    src = np.array([[24, 15], [24, 40]])
    xs = np.arange(1, nx, 4)
    rec = np.concatenate([inputs.surface_line(2, 2, xs), inputs.surface_line(2, 40, xs)], axis=1)
    nshot, nrec = src.shape[0], rec.shape[1]
    w = np.stack([inputs.ricker(f0 * (1 + 0.05 * k), dt, nt) for k in range(nshot)]) * 1e6
    p = sw.problem(sw.ELASTIC, nz=nz, nx=nx, pml=pml, dx=dx, dt=dt, nt=nt, nshot=nshot,
                   nrec=nrec, f_ref=f0, v_pml=3000.0)
    q = oracle.make_problem(1, nz, nx, pml, np.float32(dx), np.float32(dt), nt, nshot, nrec,
                            np.float32(f0), v_pml=3000.0)
    dobs = oracle.elastic_forward(q, f32(mt), f32(w), src, rec).astype(np.float32)
    mtt, wt, st, rt = _tensors(sw, m, w, src, rec)
    g, J, _ = sw.sweep_gradient(p, mtt, wt, st, rt, torch.tensor(dobs, device="cuda"))
    g = g.cpu().numpy()
    gref, Jref = oracle.elastic_gradient(q, f32(m), f32(w), src, rec, dobs.astype(np.float64))
    assert np.all(np.isfinite(g))
    assert abs(float(J) - Jref) <= 2e-3 * Jref, (float(J), Jref)
    assert np.all(gref[1][:16] == 0.0)   # no Vs sensitivity inside the fluid
    for k in range(3):
        assert np.abs(gref[k]).max() > 0
        assert rel(g[k], gref[k]) <= 1e-3, (k, rel(g[k], gref[k]))


def test_elastic_adjoint_kernels_multi_unit_vs_oracle(sw):
    """The adjoint kernels' pipeline beyond one unit per CTA: 129x333 + 11
    (30 tiles of 16 x 128, 7 of them plain: no strip, box inside the grid),
    121 shots, so the shots go in groups of 2 (61 groups, the last with one
    shot and an empty slot) and every CTA runs 24-26 (tile, shot) steps
    through its two stages; nt 60 (segments of 8, the last one short).  Receivers within 6 cells of the source, clipped to
    the grid, so that shots near an edge have several receivers on one cell
    (their residuals must add up).  Gradient per parameter and wavelet
    adjoint, whole and per shot, against the FP64 oracle."""
    nz, nx, pml, nt, nshot, nrec = 129, 333, 11, 60, 121, 7
    rng = np.random.default_rng(21)
    m = random_model(nz, nx, 21)
    src = np.stack([rng.integers(2, nz - 2, nshot), rng.integers(2, nx - 2, nshot)], -1)
    # receivers within 6 cells of their shot's source, so that every shot's
    # adjoint wave reaches its source within nt steps
    off = rng.integers(-6, 7, (nshot, nrec, 2))
    rec = np.stack([np.clip(src[:, None, 0] + off[..., 0], 0, nz - 1),
                    np.clip(src[:, None, 1] + off[..., 1], 0, nx - 1)], -1)
    dt, dx, f0 = 4e-4, 5.0, 25.0
    w = np.stack([inputs.ricker(f0 * (1 + 0.01 * (k % 7)), dt, nt) for k in range(nshot)]) * 1e6
    mt = m.copy()
    mt[0, 30:60, 20:50] *= 1.04
    mt[1, 70:100, 60:110] *= 0.95
    mt[2, 10:40, 90:120] *= 1.05
    mt[0, 60:90, 150:200] *= 0.96
    kw = dict(nz=nz, nx=nx, pml=pml, dx=dx, dt=dt, nt=nt, nshot=nshot, nrec=nrec, f_ref=f0,
              v_pml=4000.0)
    p = sw.problem(sw.ELASTIC, **kw)
    q = oracle.make_problem(1, nz, nx, pml, np.float32(dx), np.float32(dt), nt, nshot, nrec,
                            np.float32(f0), v_pml=4000.0)
    dobs = oracle.elastic_forward(q, f32(mt), f32(w), src, rec).astype(np.float32)
    mtt, wt, st, rt = _tensors(sw, m, w, src, rec)
    g, J, _ = sw.sweep_gradient(p, mtt, wt, st, rt, torch.tensor(dobs, device="cuda"))
    g = g.cpu().numpy()
    gref, Jref = oracle.elastic_gradient(q, f32(m), f32(w), src, rec, dobs.astype(np.float64))
    assert abs(float(J) - Jref) <= 2e-3 * Jref, (float(J), Jref)
    for k in range(3):
        assert np.abs(gref[k]).max() > 0
        assert rel(g[k], gref[k]) <= 1e-3, (k, rel(g[k], gref[k]))
    adj = rng.standard_normal((nshot, 2, nrec, nt)).astype(np.float32)
    wg = sw.sweep_adjoint(p, mtt, torch.tensor(adj, device="cuda"), st, rt).cpu().numpy()
    ref = oracle.elastic_adjoint(q, f32(m), adj.astype(np.float64), src, rec)
    assert rel(wg, ref) <= 1e-4, rel(wg, ref)
    per_shot = [rel(wg[s], ref[s]) for s in range(nshot)]
    assert max(per_shot) <= 1e-3, max(per_shot)


def test_elastic_gradient_is_bitwise_reproducible(sw):
    """Two identical elastic gradient calls give identical bits, on the
    multi-unit case (129x333 + 11, 121 shots in groups of 2, nt 60): the
    transposed kernels add every term in a fixed order (the coefficient
    adjoints per shot group, in shot order, then the groups in order) and
    use no atomics except the receiver injection, whose order matters only
    for receivers sharing a cell (none here)."""
    nz, nx, pml, nt, nshot, nrec = 129, 333, 11, 60, 121, 7
    rng = np.random.default_rng(31)
    m = random_model(nz, nx, 31)
    src = np.stack([rng.integers(2, nz - 2, nshot), rng.integers(2, nx - 2, nshot)], -1)
    cols = np.clip(src[:, 1:2] - 9, 0, nx - 19) + np.arange(0, 21, 3)[None, :]  # distinct
    rec = np.stack([np.clip(src[:, 0:1] - 3, 0, nz - 1).repeat(nrec, 1), cols], -1)
    assert all(len(set(map(tuple, rec[s]))) == nrec for s in range(nshot))
    dt, dx, f0 = 4e-4, 5.0, 25.0
    w = np.stack([inputs.ricker(f0, dt, nt)] * nshot) * 1e6
    p = sw.problem(sw.ELASTIC, nz=nz, nx=nx, pml=pml, dx=dx, dt=dt, nt=nt, nshot=nshot,
                   nrec=nrec, f_ref=f0, v_pml=4000.0)
    mt, wt, st, rt = _tensors(sw, m, w, src, rec)
    dobs = torch.zeros((nshot, 2, nrec, nt), device="cuda")
    g1, J1, _ = sw.sweep_gradient(p, mt, wt, st, rt, dobs)
    g2, J2, _ = sw.sweep_gradient(p, mt, wt, st, rt, dobs)
    assert torch.equal(g1, g2) and float(J1) == float(J2)
    assert float(g1.abs().max()) > 0
