"""CUDA-graph capture of library calls (sweep_capture_begin / _end,
sweep_graph_launch): a replay computes what the direct call computes, reads
its inputs at replay time, and counts its kernels; a capture broken by a
synchronising call is reported, and the stream stays usable.

Replays and direct calls are compared to 1e-5 of the largest value: the two
CPML additions of a border corner cell land in either order, so runs differ
in the last bit (that tolerance is far above it and far below any error of
the scheme); gradient and misfit as in the parity tests (1e-4)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2604_14189_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import sweep
    return sweep


def setup(sw, nz=61, nx=150, pml=12, nt=200, nshot=3, nrec=11, seed=5):
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None]
    v = np.clip(1800.0 + 1200.0 * z / (nz - 1) + 100.0 * rng.standard_normal((nz, nx)),
                1500.0, 3500.0)
    src = np.stack([np.ones(nshot), rng.integers(0, nx, nshot)], -1).astype(np.int32)
    rec = np.stack([np.full((nshot, nrec), 2), rng.integers(0, nx, (nshot, nrec))],
                   -1).astype(np.int32)
    w = np.stack([inputs.ricker(12.0, 1e-3, nt)] * nshot).astype(np.float32)
    p = sw.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=nshot, nrec=nrec,
                   f_ref=12.0)
    dev = "cuda"
    return p, dict(model=torch.tensor(v, dtype=torch.float32, device=dev),
                   wavelet=torch.tensor(w, device=dev), src=torch.tensor(src, device=dev),
                   rec=torch.tensor(rec, device=dev))


def close(a, b, tol=1e-5):
    a = a.double().cpu()
    b = b.double().cpu()
    return float((a - b).abs().max()) <= tol * float(b.abs().max())


def test_forward_replay_matches_direct_call(sw):
    p, t = setup(sw)
    s = torch.cuda.Stream()
    ws = sw.alloc_workspace(p, sw.MODE_FORWARD)
    data = torch.empty((p.nshot, 1, p.nrec, p.nt), device="cuda")
    ref = sw.sweep_forward(p, t["model"], t["wavelet"], t["src"], t["rec"])
    with sw.capture(s) as cap:
        sw.sweep_forward(p, t["model"], t["wavelet"], t["src"], t["rec"], data=data, ws=ws,
                         stream=s)
    g = cap.graph
    try:
        data.zero_()
        torch.cuda.synchronize()
        g.launch(s)
        s.synchronize()
        assert sw.status(ws, s) == sw.OK
        assert close(data, ref)
        # inputs are read at replay time: a new model written in place
        t["model"].mul_(1.05)
        ref2 = sw.sweep_forward(p, t["model"], t["wavelet"], t["src"], t["rec"])
        torch.cuda.synchronize()
        g.launch(s)
        s.synchronize()
        assert close(data, ref2)
        assert not close(ref2, ref, 1e-3)
    finally:
        g.close()


def test_gradient_replay_and_launch_count(sw):
    p, t = setup(sw, seed=9)
    vt = t["model"] * 1.03
    d_obs = sw.sweep_forward(p, vt, t["wavelet"], t["src"], t["rec"])
    ws = sw.alloc_workspace(p, sw.MODE_GRADIENT)
    grad = torch.empty((p.nz, p.nx), device="cuda")
    mis = torch.empty((), dtype=torch.float64, device="cuda")
    illum = torch.empty((p.nz, p.nx), device="cuda")
    l0 = sw.kernel_launches()
    g_ref, m_ref, i_ref = sw.sweep_gradient(p, t["model"], t["wavelet"], t["src"], t["rec"],
                                            d_obs, want_illum=True)
    direct = sw.kernel_launches() - l0
    s = torch.cuda.Stream()
    l1 = sw.kernel_launches()
    with sw.capture(s) as cap:
        sw.sweep_gradient(p, t["model"], t["wavelet"], t["src"], t["rec"], d_obs, grad=grad,
                          misfit=mis, illum=illum, ws=ws, stream=s)
    g = cap.graph
    try:
        assert sw.kernel_launches() == l1  # recorded, not launched
        assert g.kernels == direct
        for _ in range(2):
            g.launch(s)
        s.synchronize()
        assert sw.kernel_launches() - l1 == 2 * direct
        assert sw.status(ws, s) == sw.OK
        assert close(grad, g_ref, 1e-4)
        assert close(illum, i_ref, 1e-4)
        assert abs(float(mis) - float(m_ref)) <= 1e-4 * abs(float(m_ref))
    finally:
        g.close()


def test_synchronising_call_breaks_capture(sw):
    """sweep_status synchronises, which a capture forbids: the capture ends
    with ECUDA, no graph is returned, and the stream works afterwards."""
    p, t = setup(sw, nt=50)
    ws = sw.alloc_workspace(p, sw.MODE_FORWARD)
    data = torch.empty((p.nshot, 1, p.nrec, p.nt), device="cuda")
    s = torch.cuda.Stream()
    L = sw.lib()
    sp = ctypes.c_void_p(s.cuda_stream)
    torch.cuda.synchronize()
    assert L.sweep_capture_begin(sp) == sw.OK
    assert L.sweep_capture_begin(sp) == sw.EINVAL  # one capture per thread
    assert L.sweep_status(ctypes.c_void_p(ws.data_ptr()), sp) == sw.ECUDA
    h = ctypes.c_void_p(None)
    assert L.sweep_capture_end(sp, ctypes.byref(h)) == sw.ECUDA
    assert not h.value
    out = sw.sweep_forward(p, t["model"], t["wavelet"], t["src"], t["rec"], data=data, ws=ws,
                           stream=s)
    s.synchronize()
    ref = sw.sweep_forward(p, t["model"], t["wavelet"], t["src"], t["rec"])
    assert close(out, ref)


@pytest.mark.gpu
def test_deterministic_graph_replay_is_bitwise_equal(sw):
    """In deterministic mode a graph replay of sweep_gradient equals the
    direct call bit for bit."""
    nz, nx, pml, nt, ns = 50, 140, 12, 200, 3
    rng = np.random.default_rng(12)
    v = np.clip(1800.0 + 900.0 * np.arange(nz)[:, None] / nz + 80.0 *
                rng.standard_normal((nz, nx)), 1500.0, 3000.0).astype(np.float32)
    src = np.stack([np.full(ns, 2), rng.integers(0, nx, ns)], -1).astype(np.int32)
    recs = np.stack([np.full((ns, 20), 2), np.tile(np.arange(0, nx, 7)[:20], (ns, 1))],
                    -1).astype(np.int32)
    p = sw.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=ns, nrec=20,
                   f_ref=12.0, flags=sw.F_DETERMINISTIC)
    dev = "cuda"
    tv = torch.tensor(v, device=dev)
    tw = torch.tensor(np.stack([inputs.ricker(12.0, 1e-3, nt)] * ns), dtype=torch.float32,
                      device=dev)
    ts, tr = torch.tensor(src, device=dev), torch.tensor(recs, device=dev)
    d_obs = sw.sweep_forward(p, tv * 1.02, tw, ts, tr)
    ws = sw.alloc_workspace(p, sw.MODE_GRADIENT)
    g = torch.empty_like(tv)
    J = torch.empty((), dtype=torch.float64, device=dev)
    s = torch.cuda.Stream()
    with sw.capture(s) as c:
        sw.sweep_gradient(p, tv, tw, ts, tr, d_obs, grad=g, misfit=J, ws=ws, stream=s)
    c.graph.launch(s)
    s.synchronize()
    gd, Jd, _ = sw.sweep_gradient(p, tv, tw, ts, tr, d_obs)
    assert torch.equal(g, gd) and float(J) == float(Jd)
    c.graph.close()
