"""Parity of the CUDA acoustic path (through the C ABI) with the FP64 oracle.

Tolerances (stated by the solver's accuracy target):
  seismograms      relative L2 <= 1e-4
  adjoint sources  relative L2 <= 1e-4
  gradients        relative L2 <= 1e-3
  misfit           relative    <= 1e-4
  dot-product test relative    <= 1e-5 (FP64 reductions)
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_14189_gb300 import inputs
from parity_util import region_errors, worst_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import sweep
    return sweep


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def cuda(x, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)


def case(nz, nx, pml, nt, nshot, nrec, seed=0, dx=10.0, dt=1e-3, f0=15.0, flags=0,
         v_pml=0.0, src_z=None):
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None]
    v = 1800.0 + 1200.0 * z / max(nz - 1, 1) + 150.0 * rng.standard_normal((nz, nx))
    v = np.clip(v, 1500.0, 3500.0)
    sx = rng.integers(0, nx, nshot)
    sz = np.full(nshot, 1 if src_z is None else src_z)
    src = np.stack([sz, sx], -1).astype(np.int32)
    rec = np.stack([rng.integers(0, nz, (nshot, nrec)), rng.integers(0, nx, (nshot, nrec))],
                   -1).astype(np.int32)
    w = np.stack([inputs.ricker(f0 * (1 + 0.1 * k), dt, nt) for k in range(nshot)])
    return dict(nz=nz, nx=nx, pml=pml, nt=nt, nshot=nshot, nrec=nrec, dx=dx, dt=dt, f0=f0,
                v=v, src=src, rec=rec, w=w, flags=flags, v_pml=v_pml)


def probs(sw, c):
    p = sw.problem(nz=c["nz"], nx=c["nx"], pml=c["pml"], dx=c["dx"], dt=c["dt"], nt=c["nt"],
                   nshot=c["nshot"], nrec=c["nrec"], f_ref=c["f0"], v_pml=c["v_pml"],
                   flags=c["flags"])
    # the oracle sees exactly the FP32 values the GPU sees
    q = oracle.make_problem(0, c["nz"], c["nx"], c["pml"], np.float32(c["dx"]),
                            np.float32(c["dt"]), c["nt"], c["nshot"], c["nrec"],
                            np.float32(c["f0"]), c["flags"], v_pml=np.float32(c["v_pml"]))
    return p, q


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


# several tiles in x and z, ragged tails, sources next to the border
SHAPES = [
    (37, 45, 6, 300, 3, 7),
    (70, 301, 20, 400, 2, 25),
    (129, 133, 11, 250, 4, 9),
    (8, 9, 4, 120, 1, 3),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(sw, shape):
    c = case(*shape, seed=sum(shape))
    p, q = probs(sw, c)
    d = sw.sweep_forward(p, cuda(c["v"]), cuda(c["w"]), cuda(c["src"], torch.int32),
                         cuda(c["rec"], torch.int32)).cpu().numpy()[:, 0]
    ref = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"])
    assert np.abs(ref).max() > 0
    assert rel(d, ref) <= 1e-4, rel(d, ref)
    assert worst_trace(d, ref) <= 1e-3, worst_trace(d, ref)


def test_forward_without_border_and_padded_model(sw):
    c = case(40, 52, 0, 300, 2, 6, seed=3)
    p, q = probs(sw, c)
    d = sw.sweep_forward(p, cuda(c["v"]), cuda(c["w"]), cuda(c["src"], torch.int32),
                         cuda(c["rec"], torch.int32)).cpu().numpy()[:, 0]
    ref = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"])
    assert rel(d, ref) <= 1e-4
    c = case(40, 52, 9, 300, 2, 6, seed=4, flags=sw.F_PADDED_MODEL)
    vp = inputs.pad_edge(c["v"], 9)
    vp[:3] *= 1.1  # the padded values are really used
    p, q = probs(sw, c)
    d = sw.sweep_forward(p, cuda(vp), cuda(c["w"]), cuda(c["src"], torch.int32),
                         cuda(c["rec"], torch.int32)).cpu().numpy()[:, 0]
    ref = oracle.acoustic_forward(q, f32(vp), f32(c["w"]), c["src"], c["rec"])
    assert rel(d, ref) <= 1e-4


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_adjoint_matches_oracle(sw, shape):
    c = case(*shape, seed=7 + sum(shape))
    p, q = probs(sw, c)
    rng = np.random.default_rng(1)
    r = rng.standard_normal((c["nshot"], c["nrec"], c["nt"]))
    wg = sw.sweep_adjoint(p, cuda(c["v"]), cuda(r), cuda(c["src"], torch.int32),
                          cuda(c["rec"], torch.int32)).cpu().numpy()
    ref = oracle.acoustic_adjoint(q, f32(c["v"]), f32(r), c["src"], c["rec"])
    assert rel(wg, ref) <= 1e-4, rel(wg, ref)


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_gradient_matches_oracle(sw, shape):
    c = case(*shape, seed=11 + sum(shape))
    p, q = probs(sw, c)
    rng = np.random.default_rng(2)
    v_true = c["v"] * (1 + 0.03 * rng.standard_normal(c["v"].shape))
    d_obs = oracle.acoustic_forward(q, f32(v_true), f32(c["w"]), c["src"], c["rec"])
    g, J, _ = sw.sweep_gradient(p, cuda(c["v"]), cuda(c["w"]), cuda(c["src"], torch.int32),
                                cuda(c["rec"], torch.int32), cuda(d_obs))
    gref, Jref = oracle.acoustic_gradient(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"],
                                          f32(d_obs))
    # J = 1/2 |d - d_obs|^2: with |d - d_ref| <= 1e-4 |d_ref| (seismogram
    # tolerance), |J - J_ref| <= 1e-4 |d_ref| |r_ref| + 1/2 (1e-4 |d_ref|)^2
    d_ref = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"])
    nd, nr = np.linalg.norm(d_ref), np.linalg.norm(d_ref - f32(d_obs))
    assert abs(J.item() - Jref) <= 1e-4 * nd * nr + 0.5e-8 * nd ** 2
    assert rel(g.cpu().numpy(), gref) <= 1e-3, rel(g.cpu().numpy(), gref)
    errs = region_errors(g.cpu().numpy(), gref, c["src"])
    assert max(errs.values()) <= 1e-3, errs


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_16_row_tiles_match_oracle(sw, shape):
    """SWEEP_F_ROWS16 (stencil tiles of 16 rows) changes the work split only:
    forward, adjoint and gradient meet the oracle at the same tolerances and
    agree with the 32-row path to FP32 rounding (the CPML corner cells take
    two atomic additions in either order)."""
    c = case(*shape, seed=31 + sum(shape))
    p, q = probs(sw, c)
    p16, _ = probs(sw, dict(c, flags=sw.F_ROWS16))
    v, w = cuda(c["v"]), cuda(c["w"])
    src, rec = cuda(c["src"], torch.int32), cuda(c["rec"], torch.int32)
    d16 = sw.sweep_forward(p16, v, w, src, rec).cpu().numpy()[:, 0]
    d32 = sw.sweep_forward(p, v, w, src, rec).cpu().numpy()[:, 0]
    ref = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"])
    assert rel(d16, ref) <= 1e-4 and worst_trace(d16, ref) <= 1e-3
    assert rel(d16, d32) <= 1e-6, rel(d16, d32)
    rng = np.random.default_rng(3)
    r = rng.standard_normal((c["nshot"], c["nrec"], c["nt"]))
    wg = sw.sweep_adjoint(p16, v, cuda(r), src, rec).cpu().numpy()
    wref = oracle.acoustic_adjoint(q, f32(c["v"]), f32(r), c["src"], c["rec"])
    assert rel(wg, wref) <= 1e-4, rel(wg, wref)
    v_true = c["v"] * (1 + 0.03 * rng.standard_normal(c["v"].shape))
    d_obs = oracle.acoustic_forward(q, f32(v_true), f32(c["w"]), c["src"], c["rec"])
    g16, J16, _ = sw.sweep_gradient(p16, v, w, src, rec, cuda(d_obs))
    g32, J32, _ = sw.sweep_gradient(p, v, w, src, rec, cuda(d_obs))
    gref, Jref = oracle.acoustic_gradient(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"],
                                          f32(d_obs))
    g16 = g16.cpu().numpy()
    assert rel(g16, gref) <= 1e-3, rel(g16, gref)
    assert max(region_errors(g16, gref, c["src"]).values()) <= 1e-3
    assert rel(g16, g32.cpu().numpy()) <= 1e-4  # corner additions in either order
    # the misfit bound of test_gradient_matches_oracle (J is a difference of
    # nearly equal data, so its relative rounding is |d| / |r| times larger)
    nd, nr = np.linalg.norm(ref), np.linalg.norm(ref - f32(d_obs))
    assert abs(J16.item() - Jref) <= 1e-4 * nd * nr + 0.5e-8 * nd ** 2


def test_deterministic_mode_is_bitwise_reproducible(sw):
    """SWEEP_F_DETERMINISTIC: every cell has one writer per kernel phase (the
    CPML x part owns the corners of the border band and adds both axes'
    terms there; the backward stencil kernel injects the residual at the
    receivers, in receiver order), so two identical runs give bitwise equal
    seismograms, adjoint sources, gradients, misfits and illumination, in
    both tile heights, and they meet the oracle like the default mode.
    Receivers sit in the band rows, on the corners and twice on one cell.
    (The two tile heights are separate instantiations whose compiled
    arithmetic may contract differently, so they agree to FP32 rounding.)"""
    c = case(70, 301, 20, 300, 3, 25, seed=77)
    c["rec"][:, :6] = [[0, 0], [1, 300], [2, 2], [69, 0], [69, 300], [2, 2]]
    ref = oracle.acoustic_forward(probs(sw, c)[1], f32(c["v"]), f32(c["w"]), c["src"],
                                  c["rec"])
    _, q = probs(sw, c)
    v, w = cuda(c["v"]), cuda(c["w"])
    src, rec = cuda(c["src"], torch.int32), cuda(c["rec"], torch.int32)
    rng = np.random.default_rng(4)
    r = rng.standard_normal((c["nshot"], c["nrec"], c["nt"]))
    wref = oracle.acoustic_adjoint(q, f32(c["v"]), f32(r), c["src"], c["rec"])
    gref, _ = oracle.acoustic_gradient(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"],
                                       f32(ref * 1.05))
    results = {}
    for rows16 in (False, True):
        flags = sw.F_DETERMINISTIC | (sw.F_ROWS16 if rows16 else 0)
        p, _ = probs(sw, dict(c, flags=flags))
        d = [sw.sweep_forward(p, v, w, src, rec) for _ in range(2)]
        assert torch.equal(d[0], d[1])
        assert rel(d[0].cpu().numpy()[:, 0], ref) <= 1e-4
        wg = [sw.sweep_adjoint(p, v, cuda(r), src, rec) for _ in range(2)]
        assert torch.equal(wg[0], wg[1])
        assert rel(wg[0].cpu().numpy(), wref) <= 1e-4
        out = [sw.sweep_gradient(p, v, w, src, rec, cuda(ref * 1.05), want_illum=True)
               for _ in range(2)]
        assert all(torch.equal(a, b) for a, b in zip(out[0], out[1]))
        assert rel(out[0][0].cpu().numpy(), gref) <= 1e-3
        results[rows16] = (d[0], wg[0], out[0][0])
    for a, b in zip(results[False], results[True]):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-5


def test_gradient_residual_mode_and_illumination(sw):
    c = case(45, 60, 8, 260, 2, 5, seed=21, flags=0)
    p, q = probs(sw, c)
    c2 = dict(c, flags=sw.F_RESIDUAL_IN)
    p2, q2 = probs(sw, c2)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((c["nshot"], c["nrec"], c["nt"])) * 1e-3
    g, J, ill = sw.sweep_gradient(p2, cuda(c["v"]), cuda(c["w"]), cuda(c["src"], torch.int32),
                                  cuda(c["rec"], torch.int32), cuda(r), want_illum=True)
    gref, Jref = oracle.acoustic_gradient(q2, f32(c["v"]), f32(c["w"]), c["src"], c["rec"],
                                          f32(r))
    assert abs(J.item() - Jref) <= 1e-5 * Jref
    assert rel(g.cpu().numpy(), gref) <= 1e-3
    # illumination: sum over shots and n = 0 .. nt-1 of (u^n)^2 on the interior
    _, wf = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"],
                                    wavefield=True)
    P = c["pml"]
    iref = np.sum(wf[:, :c["nt"], P:P + c["nz"], P:P + c["nx"]] ** 2, axis=(0, 1))
    assert rel(ill.cpu().numpy(), iref) <= 1e-4


def test_dot_product_tests(sw):
    """<F w, d> = <w, F^T d> and <J dv, r> = <dv, J^T r>, FP64 reductions."""
    c = case(60, 90, 12, 400, 3, 11, seed=31)
    p, _ = probs(sw, c)
    rng = np.random.default_rng(8)
    w = cuda(rng.standard_normal((c["nshot"], c["nt"])))
    d = cuda(rng.standard_normal((c["nshot"], c["nrec"], c["nt"])))
    v, src, rec = cuda(c["v"]), cuda(c["src"], torch.int32), cuda(c["rec"], torch.int32)
    Fw = sw.sweep_forward(p, v, w, src, rec)
    Ftd = sw.sweep_adjoint(p, v, d, src, rec)
    lhs = sw.sweep_dot(Fw.reshape(-1), d.reshape(-1)).item()
    rhs = sw.sweep_dot(w.reshape(-1), Ftd.reshape(-1)).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
    # sweep_dot itself against an FP64 host sum
    a, b = Fw.reshape(-1), d.reshape(-1)
    ref = float(np.dot(a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)))
    assert abs(lhs - ref) <= 1e-12 * abs(ref)


def test_gradient_finite_differences(sw):
    """FD of the GPU misfit (FP64 reduction, FP32 forward) along 10 smooth
    perturbations of a padded model vs <g, dv>: within 1e-2 of the larger of
    the directional derivative and half the largest one of the set.  A
    perturbation whose derivative nearly cancels (one here is 3 % of the
    largest) carries the central difference's truncation error of the
    non-quadratic misfit (~1e-3 of the set's scale at this step) on a small
    value, so its check is against the set's scale."""
    c = case(50, 70, 10, 350, 2, 12, seed=41, flags=sw.F_PADDED_MODEL, v_pml=3600.0)
    p, _ = probs(sw, c)
    P = c["pml"]
    vpad = inputs.pad_edge(c["v"], P)
    rng = np.random.default_rng(3)
    d_obs = sw.sweep_forward(p, cuda(vpad * (1 + 0.05 * rng.standard_normal(vpad.shape))),
                             cuda(c["w"]), cuda(c["src"], torch.int32),
                             cuda(c["rec"], torch.int32))
    g, J, _ = sw.sweep_gradient(p, cuda(vpad), cuda(c["w"]), cuda(c["src"], torch.int32),
                                cuda(c["rec"], torch.int32), d_obs)
    g = g.cpu().numpy().astype(np.float64)
    pert = inputs.smooth_perturbations(c["nz"], c["nx"], c["v"], 10, seed=5, sigma=5.0)
    pairs = []
    for k in range(10):
        dv = np.zeros_like(vpad)
        dv[P:P + c["nz"], P:P + c["nx"]] = pert[k]
        h = 0.5  # the perturbation is 1 % of v; step 0.5 of it
        Js = []
        for sgn in (1, -1):
            _, Jk, _ = sw.sweep_gradient(p, cuda(vpad + sgn * h * dv), cuda(c["w"]),
                                         cuda(c["src"], torch.int32),
                                         cuda(c["rec"], torch.int32), d_obs)
            Js.append(Jk.item())
        fd = (Js[0] - Js[1]) / (2 * h)
        an = float(np.sum(g * pert[k]))
        pairs.append((fd, an))
    top = max(abs(an) for _, an in pairs)
    assert sum(abs(an) >= 0.1 * top for _, an in pairs) >= 5  # mostly non-cancelling
    for k, (fd, an) in enumerate(pairs):
        assert abs(fd - an) <= 1e-2 * max(abs(an), 0.5 * top), (k, fd, an, top)


def test_layered_single_shot_full_size(sw):
    """200 x 200 + 40-cell CPML, nt = 1000, 10 Hz, 200 receivers."""
    wl = inputs.workload_layered3()
    c = dict(nz=wl["nz"], nx=wl["nx"], pml=wl["pml"], nt=wl["nt"], nshot=1, nrec=200,
             dx=wl["dx"], dt=wl["dt"], f0=wl["f0"], flags=0, v_pml=0.0)
    p, q = probs(sw, c)
    w = inputs.ricker(wl["f0"], wl["dt"], wl["nt"])[None]
    d = sw.sweep_forward(p, cuda(wl["model"]), cuda(w), cuda(wl["src"], torch.int32),
                         cuda(wl["rec"], torch.int32)).cpu().numpy()[:, 0]
    ref = oracle.acoustic_forward(q, f32(wl["model"]), f32(w), wl["src"], wl["rec"])
    assert rel(d, ref) <= 1e-4, rel(d, ref)


def test_edge_cases(sw):
    c = case(30, 40, 5, 100, 2, 4, seed=51)
    p, q = probs(sw, c)
    v, w = cuda(c["v"]), cuda(c["w"])
    src, rec = cuda(c["src"], torch.int32), cuda(c["rec"], torch.int32)
    # no receivers: runs, returns an empty record
    p0 = sw.problem(nz=30, nx=40, pml=5, dx=10.0, dt=1e-3, nt=100, nshot=2, nrec=0)
    d = sw.sweep_forward(p0, v, w, src, torch.zeros((2, 0, 2), dtype=torch.int32, device="cuda"))
    assert d.shape == (2, 1, 0, 100)
    # no shots: gradient is zero
    pz = sw.problem(nz=30, nx=40, pml=5, dx=10.0, dt=1e-3, nt=100, nshot=0, nrec=4)
    g, J, _ = sw.sweep_gradient(pz, v, w[:0], src[:0], rec[:0],
                                torch.zeros((0, 4, 100), device="cuda"))
    assert float(g.abs().max()) == 0.0 and J.item() == 0.0
    # device-detected errors are latched and reported
    bad = c["src"].copy()
    bad[1, 1] = 40
    with pytest.raises(sw.SweepError) as e:
        sw.sweep_forward(p, v, w, cuda(bad, torch.int32), rec)
    assert e.value.code == sw.EBOUNDS
    with pytest.raises(sw.SweepError) as e:
        sw.sweep_forward(p, v * 3.0, w, src, rec)  # 5250 m/s * 1 ms / 10 m > 0.5546
    assert e.value.code == sw.ECFL
    vb = c["v"].copy()
    vb[3, 4] = np.nan
    with pytest.raises(sw.SweepError) as e:
        sw.sweep_forward(p, cuda(vb), w, src, rec)
    assert e.value.code == sw.ENONFINITE
    vb[3, 4] = -1.0
    with pytest.raises(sw.SweepError) as e:
        sw.sweep_forward(p, cuda(vb), w, src, rec)
    assert e.value.code == sw.EMODEL
    # the workspace is reusable after an error
    d = sw.sweep_forward(p, v, w, src, rec).cpu().numpy()[:, 0]
    ref = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"])
    assert rel(d, ref) <= 1e-4
    # the illumination output is acoustic only
    pe = sw.problem(sw.ELASTIC, nz=30, nx=40, pml=5, dx=10.0, dt=1e-3, nt=100, nshot=2, nrec=4)
    me = torch.stack([torch.full((30, 40), 2000.0), torch.full((30, 40), 1000.0),
                      torch.full((30, 40), 2000.0)]).cuda()
    with pytest.raises(sw.SweepError) as e:
        sw.sweep_gradient(pe, me, torch.zeros((2, 100), device="cuda"), src, rec,
                          torch.zeros((2, 2, 4, 100), device="cuda"), want_illum=True)
    assert e.value.code == sw.EUNSUPPORTED


def test_bounded_wait_runs_out_and_context_survives(sw):
    """A device-side wait that nothing completes gives up after its bound,
    latches ETIMEOUT in the status word, and leaves the context usable: the
    next call on the same workspace clears the word and matches the oracle."""
    c = case(30, 40, 5, 80, 1, 3, seed=61)
    p, q = probs(sw, c)
    ws = sw.alloc_workspace(p, sw.MODE_FORWARD)
    sw.check_wait_timeout(ws)
    assert sw.status(ws) == sw.ETIMEOUT
    d = sw.sweep_forward(p, cuda(c["v"]), cuda(c["w"]), cuda(c["src"], torch.int32),
                         cuda(c["rec"], torch.int32), ws=ws)
    ref = oracle.acoustic_forward(q, f32(c["v"]), f32(c["w"]), c["src"], c["rec"])
    assert rel(d.cpu().numpy()[:, 0], ref) <= 1e-4
