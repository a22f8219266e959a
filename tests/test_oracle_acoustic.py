"""Pins of the FP64 acoustic oracle against mathematics, not against itself.

Each test fixes a property that a plausible mistake in the oracle (a dropped
term, a wrong sign or index, a transposed operand) would break:

* stencil exactness on polynomials (coefficients of the 8th-order operators);
* the closed-form 2D Green's function of u_tt = v^2 Lap u + v^2 f delta,
  convolved with a Ricker wavelet, with second-order convergence in dt
  (interior scheme, source normalisation, record timing);
* exact conservation of the discrete energy without absorbing boundary
  (time stepping, symmetry of the Laplacian);
* the CFL limit v dt / dx <= 2 / sqrt(2 * 6.50159) of the 8th-order scheme;
* source-receiver reciprocity (symmetry of the propagator);
* absorption of the convolutional PML (energy decay, reflection);
* the adjoint equals the transpose of the dense forward matrix (brute force);
* the velocity gradient equals central finite differences of the misfit.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2604_14189_gb300 import inputs

C2 = np.array([-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560])


# ----------------------------------------------------------------- stencils
@pytest.mark.parametrize("kind,order", [(0, 2), (1, 1)])
def test_stencil_exact_on_polynomials(kind, order):
    """8th-order D2 (kind 0) is exact on x^k, k <= 9; D1 (kind 1) on k <= 8."""
    x = np.arange(40, dtype=np.float64) - 20.0
    kmax = 9 if kind == 0 else 8
    for k in range(kmax + 1):
        f = x ** k
        out = oracle.stencil_1d(kind, f)
        if order == 2:
            exact = k * (k - 1) * x ** (k - 2) if k >= 2 else 0 * x
        else:
            exact = k * x ** (k - 1) if k >= 1 else 0 * x
        sl = slice(4, -4)  # away from the zero padding
        scale = np.abs(f[sl]).max() + 1.0
        np.testing.assert_allclose(out[sl], exact[sl], atol=1e-9 * scale, rtol=0)
    # and NOT exact at the next degree (the order is 8, not higher)
    f = x ** (kmax + 1)
    out = oracle.stencil_1d(kind, f)
    if order == 2:
        exact = (kmax + 1) * kmax * x ** (kmax - 1)
    else:
        exact = (kmax + 1) * x ** kmax
    assert np.abs(out[4:-4] - exact[4:-4]).max() > 1.0


@pytest.mark.parametrize("kind", [2, 3])
def test_staggered_stencil_exact_on_polynomials(kind):
    """4th-order staggered differences are exact on x^k, k <= 4 at j +- 1/2."""
    x = np.arange(30, dtype=np.float64) - 15.0
    for k in range(5):
        out = oracle.stencil_1d(kind, x ** k)
        xe = x + 0.5 if kind == 2 else x - 0.5
        exact = k * xe ** (k - 1) if k >= 1 else 0 * x
        np.testing.assert_allclose(out[3:-3], exact[3:-3], atol=1e-9 * 15 ** k, rtol=0)


def test_nyquist_symbol_and_cfl_bound():
    """Symbol of D2 at the Nyquist wavenumber = -6.50159 (sets the CFL limit)."""
    n = 64
    f = (-1.0) ** np.arange(n)
    out = oracle.stencil_1d(0, f)
    sym = out[10:-10] / f[10:-10]
    np.testing.assert_allclose(sym, -6.501587301587, rtol=1e-12)
    assert abs(2 / np.sqrt(2 * 6.501587301587) - 0.5546325) < 1e-6


# ------------------------------------------------------------ Green's function
def _green_trace(f, r, v, ts):
    """u(r, t) = (1 / 2 pi) int_0^{acosh(vt/r)} f(t - (r/v) cosh s) ds, the
    2D free-space solution of u_tt = v^2 Lap u + v^2 f(t) delta(x)."""
    out = np.zeros_like(ts)
    for k, t in enumerate(ts):
        if v * t > r:
            val, _ = integrate.quad(lambda s: f(t - (r / v) * np.cosh(s)), 0.0,
                                    np.arccosh(v * t / r), limit=200)
            out[k] = val / (2 * np.pi)
    return out


def test_green_function_convergence(golden):
    """The paper's acoustic example setting (Sec. 3.1.3: homogeneous 2000 m/s,
    20 Hz Ricker at the centre, from tests/golden/acoustic_example.json);
    trace 200 m away."""
    ex = golden("acoustic_example.json")
    assert ex["source"] == "centre"
    f0, v, dx, T = ex["ricker_peak_hz"], ex["vp_m_s"], 5.0, 0.2
    n = 161
    errs = []
    for dt in (5e-4, 2.5e-4):
        nt = int(round(T / dt))
        p = oracle.make_problem(0, n, n, 0, dx, dt, nt, 1, 1, f0)
        src = np.array([[80, 80]])
        rec = np.array([[[80, 120]]])
        d = oracle.acoustic_forward(p, np.full((n, n), v), inputs.ricker(f0, dt, nt)[None],
                                    src, rec)[0, 0]
        ts = (np.arange(nt) + 1) * dt  # trace sample n is u^{n+1}
        rk = lambda t: inputs.ricker(f0, 1.0, 1, shift=t)[0]
        a = _green_trace(rk, 40 * dx, v, ts)
        errs.append(np.linalg.norm(d - a) / np.linalg.norm(a))
    assert errs[0] < 8e-3, errs
    assert errs[1] < 2.5e-3, errs
    order = np.log2(errs[0] / errs[1])
    assert 1.7 < order < 2.3, (errs, order)


# ----------------------------------------------------------------- energy
def _lap(u):
    """Zero-padded 8th-order 5-point-per-axis Laplacian (unit spacing)."""
    out = 2 * C2[0] * u
    up = np.pad(u, 4)
    nz, nx = u.shape
    for k in range(1, 5):
        out += C2[k] * (up[4 + k:4 + k + nz, 4:4 + nx] + up[4 - k:4 - k + nz, 4:4 + nx]
                        + up[4:4 + nz, 4 + k:4 + k + nx] + up[4:4 + nz, 4 - k:4 - k + nx])
    return out


def test_energy_conserved_without_pml():
    """E^{n+1/2} = sum (u^{n+1}-u^n)^2 / K - sum u^{n+1} L u^n is constant
    once the source has stopped (random heterogeneous model, Dirichlet)."""
    rng = np.random.default_rng(7)
    nz, nx, nt, dx, dt = 40, 50, 400, 10.0, 1e-3
    v = rng.uniform(1500, 3000, (nz, nx))
    K = v ** 2 * dt ** 2 / dx ** 2
    w = np.zeros(nt)
    w[:30] = inputs.ricker(25.0, dt, 30)  # source stops after 30 steps
    p = oracle.make_problem(0, nz, nx, 0, dx, dt, nt, 1, 1, 10.0)
    _, wf = oracle.acoustic_forward(p, v, w[None], np.array([[20, 25]]),
                                    np.array([[[5, 5]]]), wavefield=True)
    u = wf[0]
    E = [np.sum((u[n + 1] - u[n]) ** 2 / K) - np.sum(u[n + 1] * _lap(u[n]))
         for n in range(31, nt)]
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() / E[0] < 1e-12


def test_energy_decays_with_cpml():
    """With a 20-cell CPML the field leaves the box: energy after 3 crossing
    times is < 1e-3 of its peak, after 2000 steps < 1e-4, with no late growth."""
    nz = nx = 60
    dx, dt, v = 10.0, 1e-3, 2000.0
    nt = 2000
    w = np.zeros(nt)
    w[:150] = inputs.ricker(10.0, dt, 150)
    p = oracle.make_problem(0, nz, nx, 20, dx, dt, nt, 1, 1, 10.0)
    _, wf = oracle.acoustic_forward(p, np.full((nz, nx), v), w[None],
                                    np.array([[30, 30]]), np.array([[[0, 0]]]),
                                    wavefield=True)
    e = np.array([np.sum(x ** 2) for x in wf[0]])  # whole padded grid
    assert np.all(np.isfinite(e))
    crossing = int(nx * dx / v / dt)
    assert e[150 + 3 * crossing] < 1e-3 * e.max()
    assert e[-1] < 1e-4 * e.max()
    assert e[-1] < e[1000]


def test_cpml_reflection_below_one_percent():
    """Trace near the boundary vs the same trace on a 3x larger domain."""
    dx, dt, v, f0, nt = 10.0, 1e-3, 2000.0, 10.0, 700
    w = inputs.ricker(f0, dt, nt)[None]
    n1 = 80
    p1 = oracle.make_problem(0, n1, n1, 30, dx, dt, nt, 1, 1, f0)
    d1 = oracle.acoustic_forward(p1, np.full((n1, n1), v), w, np.array([[40, 40]]),
                                 np.array([[[40, 70]]]))[0, 0]
    n2 = 3 * n1
    off = n1
    p2 = oracle.make_problem(0, n2, n2, 30, dx, dt, nt, 1, 1, f0)
    d2 = oracle.acoustic_forward(p2, np.full((n2, n2), v), w,
                                 np.array([[40 + off, 40 + off]]),
                                 np.array([[[40 + off, 70 + off]]]))[0, 0]
    direct = np.abs(d2).max()
    refl = np.abs(d1 - d2).max()
    assert refl < 0.01 * direct, refl / direct


# ----------------------------------------------------------------- CFL
@pytest.mark.parametrize("factor,stable", [(0.99, True), (1.05, False)])
def test_cfl_limit(factor, stable):
    n, dx, v = 30, 10.0, 2000.0
    dt = factor * 0.5546325 * dx / v
    nt = 2000
    rng = np.random.default_rng(3)
    w = np.zeros(nt)
    w[:5] = rng.standard_normal(5)
    p = oracle.make_problem(0, n, n, 0, dx, dt, nt, 1, 1, 10.0)
    d = oracle.acoustic_forward(p, np.full((n, n), v), w[None], np.array([[15, 15]]),
                                np.array([[[10, 12]]]))[0, 0]
    early = np.abs(d[:50]).max()
    late = np.abs(d[-200:]).max() if np.all(np.isfinite(d[-200:])) else np.inf
    if stable:
        assert late < 10 * early
    else:
        assert late > 1e6 * early


# ------------------------------------------------------------- reciprocity
def test_reciprocity_without_pml():
    rng = np.random.default_rng(11)
    nz, nx, nt, dx, dt = 36, 44, 300, 10.0, 1e-3
    v = rng.uniform(1500, 3500, (nz, nx))
    w = inputs.ricker(15.0, dt, nt)[None]
    A, B = [7, 9], [25, 33]
    p = oracle.make_problem(0, nz, nx, 0, dx, dt, nt, 1, 1, 15.0)
    dab = oracle.acoustic_forward(p, v, w, np.array([A]), np.array([[B]]))[0, 0]
    dba = oracle.acoustic_forward(p, v, w, np.array([B]), np.array([[A]]))[0, 0]
    assert np.abs(dab).max() > 0
    np.testing.assert_allclose(dab, dba, rtol=0, atol=1e-12 * np.abs(dab).max())


def test_reciprocity_with_pml_approximate():
    rng = np.random.default_rng(12)
    nz, nx, nt, dx, dt = 36, 44, 400, 10.0, 1e-3
    v = rng.uniform(1500, 3500, (nz, nx))
    w = inputs.ricker(15.0, dt, nt)[None]
    A, B = [7, 9], [25, 33]
    p = oracle.make_problem(0, nz, nx, 10, dx, dt, nt, 1, 1, 15.0)
    dab = oracle.acoustic_forward(p, v, w, np.array([A]), np.array([[B]]))[0, 0]
    dba = oracle.acoustic_forward(p, v, w, np.array([B]), np.array([[A]]))[0, 0]
    assert np.linalg.norm(dab - dba) / np.linalg.norm(dab) < 2e-2


# ------------------------------------------------------- brute-force adjoint
def _tiny(nshot=2, nrec=3, pml=4, nt=30, flags=0):
    rng = np.random.default_rng(5)
    nz = nx = 12
    v = rng.uniform(1800, 3200, (nz, nx))
    src = np.array([[1, 2], [10, 9]])[:nshot]
    rec = np.array([[[0, 0], [5, 11], [11, 6]], [[3, 3], [0, 10], [11, 0]]])[:nshot, :nrec]
    # the CPML reference velocity is fixed, so the profile does not move with v
    p = oracle.make_problem(0, nz, nx, pml, 10.0, 1e-3, nt, nshot, nrec, 15.0, flags,
                            v_pml=3200.0)
    return p, v, src, rec


def test_adjoint_equals_dense_transpose():
    """Assemble F (wavelet -> data) column by column with unit wavelets and
    compare with the oracle's adjoint applied to unit data vectors."""
    p, v, src, rec = _tiny()
    S, R, nt = p.nshot, p.nrec, p.nt
    F = np.zeros((S * R * nt, S * nt))
    for col in range(S * nt):
        w = np.zeros(S * nt)
        w[col] = 1.0
        F[:, col] = oracle.acoustic_forward(p, v, w.reshape(S, nt), src, rec).ravel()
    assert np.abs(F).max() > 0
    # the PML is reached within nt steps: strips are exercised
    FT = np.zeros((S * nt, S * R * nt))
    for row in range(S * R * nt):
        e = np.zeros(S * R * nt)
        e[row] = 1.0
        FT[:, row] = oracle.acoustic_adjoint(p, v, e.reshape(S, R, nt), src, rec).ravel()
    np.testing.assert_allclose(FT, F.T, rtol=0, atol=1e-12 * np.abs(F).max())


def test_adjoint_reaches_pml():
    """The tiny adjoint problem really exercises the CPML: changing the border
    width changes the data."""
    p, v, src, rec = _tiny()
    w = inputs.ricker(15.0, 1e-3, p.nt)[None].repeat(2, 0)
    d4 = oracle.acoustic_forward(p, v, w, src, rec)
    p0 = oracle.make_problem(0, 12, 12, 0, 10.0, 1e-3, p.nt, 2, 3, 15.0)
    d0 = oracle.acoustic_forward(p0, v, w, src, rec)
    assert np.abs(d4 - d0).max() > 1e-3 * np.abs(d4).max()


def test_gradient_matches_central_differences_all_cells():
    """dJ/dv on every interior cell of a tiny grid vs central differences
    (padding frozen: the model is passed padded and only interior cells move)."""
    p, v, src, rec = _tiny(flags=oracle.F_PADDED_MODEL)
    nt = p.nt
    w = np.stack([inputs.ricker(15.0, 1e-3, nt), inputs.ricker(12.0, 1e-3, nt)])
    vpad = inputs.pad_edge(v, p.pml)
    rng = np.random.default_rng(9)
    d_obs = oracle.acoustic_forward(p, vpad * (1 + 0.05 * rng.standard_normal(vpad.shape)),
                                    w, src, rec)
    g, J = oracle.acoustic_gradient(p, vpad, w, src, rec, d_obs)

    def misfit(m):
        d = oracle.acoustic_forward(p, m, w, src, rec)
        return 0.5 * np.sum((d - d_obs) ** 2)

    assert abs(misfit(vpad) - J) <= 1e-12 * J
    h = 1e-2
    fd = np.zeros_like(g)
    P = p.pml
    for i in range(p.nz):
        for j in range(p.nx):
            mp = vpad.copy(); mp[i + P, j + P] += h
            mm = vpad.copy(); mm[i + P, j + P] -= h
            fd[i, j] = (misfit(mp) - misfit(mm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=2e-6 * np.abs(fd).max())


def test_gradient_residual_mode_is_jacobian_transpose():
    """With the residual passed in, grad = J^T r: check <J dv, r> = <dv, J^T r>
    with J dv from central differences of the forward map."""
    p, v, src, rec = _tiny(flags=oracle.F_PADDED_MODEL | oracle.F_RESIDUAL_IN)
    nt = p.nt
    w = np.stack([inputs.ricker(15.0, 1e-3, nt)] * 2)
    vpad = inputs.pad_edge(v, p.pml)
    rng = np.random.default_rng(21)
    r = rng.standard_normal((p.nshot, p.nrec, nt))
    g, J = oracle.acoustic_gradient(p, vpad, w, src, rec, r)
    assert abs(J - 0.5 * np.sum(r ** 2)) < 1e-9 * J
    dv = np.zeros_like(vpad)
    dv[p.pml:-p.pml, p.pml:-p.pml] = rng.standard_normal((p.nz, p.nx))
    h = 1e-3
    pf = oracle.make_problem(0, p.nz, p.nx, p.pml, p.dx, p.dt, nt, p.nshot, p.nrec,
                             p.f_ref, oracle.F_PADDED_MODEL, v_pml=p.v_pml)
    jd = (oracle.acoustic_forward(pf, vpad + h * dv, w, src, rec)
          - oracle.acoustic_forward(pf, vpad - h * dv, w, src, rec)) / (2 * h)
    lhs = np.sum(jd * r)
    rhs = np.sum(dv[p.pml:-p.pml, p.pml:-p.pml] * g)
    assert abs(lhs - rhs) < 1e-7 * abs(lhs)


def test_checkpointed_gradient_independent_of_segmenting():
    """nt = 30 (segments of 6) and the same run through nt = 31 truncated: the
    gradient over the first steps must not depend on segment boundaries;
    a long-run gradient equals the sum of single-shot gradients."""
    p, v, src, rec = _tiny(nt=45)
    w = np.stack([inputs.ricker(15.0, 1e-3, p.nt)] * 2)
    d_obs = np.zeros((p.nshot, p.nrec, p.nt))
    g, J = oracle.acoustic_gradient(p, v, w, src, rec, d_obs)
    gs, Js = np.zeros_like(g), 0.0
    for s in range(2):
        ps = oracle.make_problem(0, p.nz, p.nx, p.pml, p.dx, p.dt, p.nt, 1, p.nrec, p.f_ref,
                                 v_pml=p.v_pml)
        g1, J1 = oracle.acoustic_gradient(ps, v, w[s:s + 1], src[s:s + 1], rec[s:s + 1],
                                          d_obs[s:s + 1])
        gs += g1
        Js += J1
    np.testing.assert_allclose(g, gs, rtol=1e-12, atol=1e-15 * np.abs(g).max())
    assert abs(J - Js) < 1e-12 * J


def test_rejects_bad_positions():
    p, v, src, rec = _tiny()
    bad = src.copy(); bad[0, 1] = p.nx
    with pytest.raises(ValueError):
        oracle.acoustic_forward(p, v, np.zeros((2, p.nt)), bad, rec)
