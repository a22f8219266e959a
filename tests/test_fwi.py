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
