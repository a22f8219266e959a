"""FWI loop: the line search and preconditioner as host logic (CPU), and a
small acoustic inversion through the C ABI (GPU)."""
import numpy as np
import pytest
import torch

from paper_2604_14189_gb300 import fwi, inputs


def test_line_search_accepts_first_improving_step():
    target = torch.tensor([3.0, -2.0])

    def misfit(m):
        return float(((m - target) ** 2).sum())

    m0 = torch.zeros(2)
    d = torch.tensor([1.0, -1.0])
    # step 8 overshoots (J = 25 + 36 > 13), 4 improves (J = 1 + 4 = 5)
    m, j, step, trials, ok = fwi.line_search(misfit, m0, d, misfit(m0), 8.0, 5, -100, 100)
    assert ok and trials == 2 and step == 4.0
    assert torch.equal(m, torch.tensor([4.0, -4.0])) and j == 5.0


def test_line_search_keeps_model_when_nothing_improves():
    def misfit(m):
        return float((m ** 2).sum())

    m0 = torch.zeros(3)
    m, j, step, trials, ok = fwi.line_search(misfit, m0, torch.ones(3), 0.0, 1.0, 3, -1, 1)
    assert not ok and trials == 4 and j == 0.0 and torch.equal(m, m0)
    assert step == 1.0 / 16


def test_line_search_respects_bounds():
    seen = []

    def misfit(m):
        seen.append(m.clone())
        return -float(m.sum())

    m, j, step, trials, ok = fwi.line_search(misfit, torch.full((4,), 1900.0),
                                             torch.ones(4), 0.0, 500.0, 2, 1500.0, 2000.0)
    assert ok and torch.all(m == 2000.0)
    assert all(float(t.max()) <= 2000.0 for t in seen)


def test_precondition_divides_by_stabilised_illumination():
    g = torch.tensor([[2.0, -4.0], [1.0, 0.0]])
    illum = torch.tensor([[1.0, 3.0], [0.0, 9.0]])
    d = fwi.precondition(g, illum, 0.1)
    raw = -g / (illum + 0.9)
    assert torch.allclose(d, raw / raw.abs().max())
    assert float(d.abs().max()) == 1.0


class _Quadratic:
    """Stand-in for the solver in Fwi.run (CPU): J = 1/2 |m - m*|^2 with a
    non-uniform illumination, counting gradient evaluations."""

    def __init__(self):
        g = torch.Generator().manual_seed(5)
        self.target = 2000.0 + 300.0 * torch.rand(6, 7, generator=g)
        self.illum = 0.5 + torch.rand(6, 7, generator=g)
        self.calls = 0

    def misfit(self, m):
        return 0.5 * float(((m.double() - self.target.double()) ** 2).sum())

    def gradient(self, m):
        self.calls += 1
        return (m - self.target), self.misfit(m), self.illum.clone()


def _fake_fwi(q):
    f = object.__new__(fwi.Fwi)  # no solver: Fwi.run calls only these two
    f.gradient, f.misfit = q.gradient, q.misfit
    return f


def _strip_times(history):
    return [{k: v for k, v in h.items() if k != "seconds"} for h in history]


def test_checkpoint_resume_equals_uninterrupted_run(tmp_path):
    cfg = fwi.FwiConfig(iterations=6, step=40.0, vmin=1500.0, vmax=3000.0)
    m0 = torch.full((6, 7), 2100.0)
    q = _Quadratic()
    ref, href = _fake_fwi(q).run(m0, cfg)
    assert q.calls == 6 and href[-1]["misfit_after"] < href[0]["misfit"]

    ck = str(tmp_path / "state")
    q1 = _Quadratic()
    m3, h3 = _fake_fwi(q1).run(m0, fwi.FwiConfig(**{**cfg.__dict__, "iterations": 3}),
                               checkpoint=ck)
    assert q1.calls == 3 and len(h3) == 3
    q2 = _Quadratic()
    m6, h6 = _fake_fwi(q2).run(m0, cfg, checkpoint=ck)
    assert q2.calls == 3  # the three iterations already done are not repeated
    assert torch.equal(m6, ref)
    assert _strip_times(h6) == _strip_times(href)
    # a finished run resumes to itself without any solver call
    q3 = _Quadratic()
    m6b, _ = _fake_fwi(q3).run(m0, cfg, checkpoint=ck)
    assert q3.calls == 0 and torch.equal(m6b, ref)


def test_checkpoint_survives_a_crash_after_saving(tmp_path):
    cfg = fwi.FwiConfig(iterations=5, step=40.0, vmin=1500.0, vmax=3000.0)
    m0 = torch.full((6, 7), 2100.0)
    ref, href = _fake_fwi(_Quadratic()).run(m0, cfg)
    ck = str(tmp_path / "state")

    def crash(it, model, rec):
        if it == 2:
            raise RuntimeError("host died")
    with pytest.raises(RuntimeError, match="host died"):
        _fake_fwi(_Quadratic()).run(m0, cfg, callback=crash, checkpoint=ck)
    model, done, step, hist = fwi.load_state(ck)
    assert done == 3 and len(hist) == 3
    m, h = _fake_fwi(_Quadratic()).run(m0, cfg, checkpoint=ck)
    assert torch.equal(m, ref) and _strip_times(h) == _strip_times(href)


def test_load_state_rejects_what_it_cannot_resume(tmp_path):
    assert fwi.load_state(str(tmp_path / "none")) is None
    ck = str(tmp_path / "s")
    fwi.save_state(ck, torch.zeros(2, 3), 1, 10.0, [])
    model, done, step, hist = fwi.load_state(ck)
    assert model.shape == (2, 3) and done == 1 and step == 10.0 and hist == []
    with pytest.raises(ValueError, match="shape"):
        _fake_fwi(_Quadratic()).run(torch.zeros(6, 7), fwi.FwiConfig(iterations=2),
                                    checkpoint=ck)
    import json
    import os
    path = os.path.join(ck, "state.json")
    st = json.load(open(path))
    st["version"] = 99
    json.dump(st, open(path, "w"))
    with pytest.raises(ValueError, match="version"):
        fwi.load_state(ck)


def _small_case():
    from paper_2604_14189_gb300 import sweep
    from scipy.ndimage import gaussian_filter

    nz, nx, pml, dx, dt, nt, f0 = 60, 90, 20, 10.0, 1e-3, 700, 10.0
    z = np.arange(nz)[:, None] + np.zeros((1, nx))
    vt = np.where(z < 20, 1800.0, np.where(z < 40, 2300.0, 2800.0))
    vt[28:38, 35:55] += 250.0
    v0 = gaussian_filter(vt, 6.0, mode="nearest")
    nshot = 6
    sx = np.round(np.linspace(2, nx - 3, nshot)).astype(np.int32)
    src = np.stack([np.full(nshot, 2), sx], -1).astype(np.int32)
    rec = inputs.surface_line(nshot, 2, np.arange(0, nx, 2))
    dev = "cuda"
    p = sweep.problem(nz=nz, nx=nx, pml=pml, dx=dx, dt=dt, nt=nt, nshot=nshot,
                      nrec=rec.shape[1], f_ref=f0, v_pml=3500.0)
    wav = torch.tensor(np.stack([inputs.ricker(f0, dt, nt)] * nshot), dtype=torch.float32,
                       device=dev)
    src_t = torch.tensor(src, device=dev)
    rec_t = torch.tensor(rec, device=dev)
    d_obs = sweep.sweep_forward(p, torch.tensor(vt, dtype=torch.float32, device=dev), wav,
                                src_t, rec_t)
    return p, wav, src_t, rec_t, d_obs, vt, v0


@pytest.mark.gpu
def test_small_acoustic_fwi_reduces_misfit_and_model_error():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p, wav, src_t, rec_t, d_obs, vt, v0 = _small_case()
    dev = "cuda"
    inv = fwi.Fwi(p, wav, src_t, rec_t, d_obs)
    m0 = torch.tensor(v0, dtype=torch.float32, device=dev)
    cfg = fwi.FwiConfig(iterations=8, step=60.0, vmin=1500.0, vmax=3500.0)
    model, hist = inv.run(m0, cfg)
    js = [h["misfit"] for h in hist]
    assert all(h["accepted"] for h in hist)
    assert all(b < a for a, b in zip(js, js[1:]))
    assert hist[-1]["misfit_after"] < 0.5 * js[0]
    vt_t = torch.tensor(vt, dtype=torch.float32, device=dev)
    e0 = float((m0 - vt_t).norm() / vt_t.norm())
    e1 = float((model - vt_t).norm() / vt_t.norm())
    assert e1 < e0
    # the misfit of the final model, recomputed, matches the line search's value
    # (to rounding: the two CPML axes add into corner cells in either order,
    # and the misfit is a difference of FP64 sums of the traces)
    assert abs(inv.misfit(model) - hist[-1]["misfit_after"]) <= 1e-4 * hist[-1]["misfit_after"]


@pytest.mark.gpu
def test_graph_replay_fwi_matches_direct_calls():
    """The recorded-graph evaluations give the direct calls' iterations:
    same accepted steps, misfits and models to rounding (corner cells of
    the border take their two CPML additions in either order)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p, wav, src_t, rec_t, d_obs, vt, v0 = _small_case()
    m0 = torch.tensor(v0, dtype=torch.float32, device="cuda")
    cfg = fwi.FwiConfig(iterations=3, step=60.0, vmin=1500.0, vmax=3500.0)
    direct = fwi.Fwi(p, wav, src_t, rec_t, d_obs, graphs=False)
    graph = fwi.Fwi(p, wav, src_t, rec_t, d_obs, graphs=True)
    try:
        m_d, h_d = direct.run(m0, cfg)
        m_g, h_g = graph.run(m0, cfg)
        assert len(h_d) == len(h_g)
        for a, b in zip(h_d, h_g):
            assert a["trials"] == b["trials"] and a["step"] == b["step"]
            assert abs(a["misfit"] - b["misfit"]) <= 1e-4 * a["misfit"]
            assert abs(a["misfit_after"] - b["misfit_after"]) <= 1e-4 * a["misfit_after"]
        assert float((m_d - m_g).abs().max()) <= 1e-5 * float(m_d.abs().max())
        # evaluations return new tensors, not the recorded buffers
        g1, _, _ = graph.gradient(m0)
        g2, _, _ = graph.gradient(m_g)
        assert g1.data_ptr() != g2.data_ptr()
    finally:
        graph.close()
