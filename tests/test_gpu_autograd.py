"""torch.autograd.Function over the C ABI: gradients of arbitrary losses of
the seismograms with respect to velocity and wavelets, checked against the
FP64 oracle, by the dot-product test, by the direct gradient call and by
finite differences along 10 random smooth perturbations."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_14189_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import autograd, sweep
    nz, nx, nt, pml = 50, 80, 400, 12
    rng = np.random.default_rng(3)
    z = np.arange(nz)[:, None]
    v = np.clip(1800 + 1000 * z / nz + 100 * rng.standard_normal((nz, nx)), 1500, 3200)
    src = np.array([[2, 10], [2, 40], [2, 70]], dtype=np.int32)
    rec = inputs.surface_line(3, 2, np.arange(0, nx, 4))
    w = np.stack([inputs.ricker(12.0, 1e-3, nt)] * 3)
    p = sweep.problem(nz=nz, nx=nx, pml=pml, dx=10.0, dt=1e-3, nt=nt, nshot=3,
                      nrec=rec.shape[1], f_ref=12.0, v_pml=3500.0)
    dev = "cuda"
    t = dict(v=torch.tensor(v, dtype=torch.float32, device=dev),
             w=torch.tensor(w, dtype=torch.float32, device=dev),
             src=torch.tensor(src, device=dev), rec=torch.tensor(rec, device=dev))
    d_obs = sweep.sweep_forward(p, t["v"] * 1.03, t["w"], t["src"], t["rec"])
    return sweep, autograd, p, t, d_obs


def test_l2_loss_gradient_equals_gradient_call(env):
    sw, ag, p, t, d_obs = env
    v = t["v"].clone().requires_grad_(True)
    d = ag.acoustic_modelling(v, t["w"], p, t["src"], t["rec"])
    loss = 0.5 * ((d - d_obs).double() ** 2).sum()
    loss.backward()
    g, J, _ = sw.sweep_gradient(p, t["v"], t["w"], t["src"], t["rec"], d_obs)
    assert abs(loss.item() - J.item()) <= 1e-6 * J.item()
    rel = (v.grad - g).norm() / g.norm()
    assert rel.item() <= 1e-5


def test_dot_product_through_autograd(env):
    sw, ag, p, t, _ = env
    torch.manual_seed(1)
    w = torch.randn_like(t["w"]).requires_grad_(True)
    y = torch.randn((p.nshot, 1, p.nrec, p.nt), device="cuda")
    d = ag.acoustic_modelling(t["v"], w, p, t["src"], t["rec"])
    lhs = (d.double() * y.double()).sum()
    (gw,) = torch.autograd.grad(lhs, w)
    rhs = (w.detach().double() * gw.double()).sum()
    assert abs(lhs.item() - rhs.item()) <= 1e-5 * abs(lhs.item())


def test_nonquadratic_loss_finite_differences(env):
    """L = sum(d^4) (smooth, not quadratic): velocity and wavelet gradients
    vs fourth-order central differences."""
    sw, ag, p, t, _ = env

    def loss_of(v, w):
        d = ag.acoustic_modelling(v, w, p, t["src"], t["rec"]).double()
        return (d * d * d * d).sum() * 1e8

    v = t["v"].clone().requires_grad_(True)
    w = t["w"].clone().requires_grad_(True)
    L = loss_of(v, w)
    gv, gw = torch.autograd.grad(L, (v, w))
    rng = np.random.default_rng(2)
    pert = inputs.smooth_perturbations(p.nz, p.nx, t["v"].cpu().numpy(), 2, seed=6, sigma=4.0)
    # the gradient holds the edge-replicated border fixed: perturb only cells
    # away from the interior edge so that the finite difference does too
    tz = np.minimum(np.arange(p.nz), np.arange(p.nz)[::-1])
    tx = np.minimum(np.arange(p.nx), np.arange(p.nx)[::-1])
    taper = np.clip(np.minimum(tz[:, None], tx[None, :]) / 6.0 - 0.5, 0.0, 1.0)
    pert = pert * taper
    for k in range(2):
        dv = torch.tensor(pert[k], dtype=torch.float32, device="cuda")
        h = 0.5
        with torch.no_grad():
            # fourth-order central difference (the loss is far from quadratic)
            f = [loss_of(t["v"] + j * h * dv, t["w"]) for j in (-2, -1, 1, 2)]
            fd = (8 * (f[2] - f[1]) - (f[3] - f[0])) / (12 * h)
        an = (gv.double() * dv.double()).sum()
        assert abs(fd.item() - an.item()) <= 2e-2 * abs(an.item()), (fd.item(), an.item())
    # the loss is a quartic of the wavelet: the stencil is exact up to rounding
    dw = torch.tensor(rng.standard_normal(t["w"].shape) * 2e-3, dtype=torch.float32,
                      device="cuda")
    with torch.no_grad():
        f = [loss_of(t["v"], t["w"] + j * dw) for j in (-2, -1, 1, 2)]
        fd = (8 * (f[2] - f[1]) - (f[3] - f[0])) / 12
    an = (gw.double() * dw.double()).sum()
    assert abs(fd.item() - an.item()) <= 2e-2 * abs(an.item()), (fd.item(), an.item())


def _taper(nz, nx, width=6.0):
    """1 away from the interior edge, 0 on it: the gradient holds the
    edge-replicated border fixed, so finite differences must not move it."""
    tz = np.minimum(np.arange(nz), np.arange(nz)[::-1])
    tx = np.minimum(np.arange(nx), np.arange(nx)[::-1])
    return np.clip(np.minimum(tz[:, None], tx[None, :]) / width - 0.5, 0.0, 1.0)


def test_autograd_l2_gradient_matches_oracle(env):
    """loss = 1/2 |d - d_obs|^2 through AcousticModelling, backward(): the
    velocity gradient against the FP64 oracle's (relative L2 <= 1e-3) and
    the loss against the oracle's misfit."""
    sw, ag, p, t, _ = env
    q = oracle.make_problem(0, p.nz, p.nx, p.pml, np.float32(p.dx), np.float32(p.dt), p.nt,
                            p.nshot, p.nrec, np.float32(p.f_ref), v_pml=np.float32(p.v_pml))
    v64 = t["v"].double().cpu().numpy()
    w64 = t["w"].double().cpu().numpy()
    src, rec = t["src"].cpu().numpy(), t["rec"].cpu().numpy()
    # observed data from the oracle (a model 3 % faster), rounded to FP32
    dob = np.float32(oracle.acoustic_forward(q, np.float32(v64 * 1.03).astype(np.float64),
                                             w64, src, rec)).astype(np.float64)
    d_obs = torch.tensor(dob[:, None], dtype=torch.float32, device="cuda")
    v = t["v"].clone().requires_grad_(True)
    d = ag.acoustic_modelling(v, t["w"], p, t["src"], t["rec"])
    loss = 0.5 * ((d - d_obs).double() ** 2).sum()
    loss.backward()
    gref, Jref = oracle.acoustic_gradient(q, v64, w64, src, rec, dob)
    g = v.grad.double().cpu().numpy()
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-3
    d_ref = oracle.acoustic_forward(q, v64, w64, src, rec)
    nd, nr = np.linalg.norm(d_ref), np.linalg.norm(d_ref - dob)
    assert abs(loss.item() - Jref) <= 1e-4 * nd * nr + 0.5e-8 * nd ** 2


def test_autograd_l2_finite_differences_ten_perturbations(env):
    """Central differences of the L2 loss (FP64 sum of FP32 records) along
    10 seeded smooth perturbations (1 % of v, tapered to zero at the
    interior edge) against <grad, dv> from backward(): within 1e-2 of the
    larger of the directional derivative and half the largest of the set
    (a derivative that nearly cancels carries the central difference's
    truncation error of the non-quadratic misfit on a small value)."""
    sw, ag, p, t, d_obs = env

    def loss_of(v):
        d = ag.acoustic_modelling(v, t["w"], p, t["src"], t["rec"])
        return 0.5 * ((d - d_obs).double() ** 2).sum()

    v = t["v"].clone().requires_grad_(True)
    (gv,) = torch.autograd.grad(loss_of(v), v)
    pert = inputs.smooth_perturbations(p.nz, p.nx, t["v"].cpu().numpy(), 10, seed=14,
                                       sigma=5.0) * _taper(p.nz, p.nx)
    pairs = []
    for k in range(10):
        dv = torch.tensor(pert[k], dtype=torch.float32, device="cuda")
        h = 0.5
        with torch.no_grad():
            fd = (loss_of(t["v"] + h * dv) - loss_of(t["v"] - h * dv)) / (2 * h)
        pairs.append((fd.item(), (gv.double() * dv.double()).sum().item()))
    top = max(abs(an) for _, an in pairs)
    assert sum(abs(an) >= 0.1 * top for _, an in pairs) >= 5
    for k, (fd, an) in enumerate(pairs):
        assert abs(fd - an) <= 1e-2 * max(abs(an), 0.5 * top), (k, fd, an, top)
