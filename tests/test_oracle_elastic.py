"""Pins of the FP64 elastic (velocity-stress, staggered) oracle.

* exact conservation of the staggered-leapfrog energy
  E^n = 1/2 <v^{n+1/2}, M v^{n-1/2}> + 1/2 <tau^n, C^{-1} tau^n>
  without absorbing boundary (operators, averaging, Hooke's law);
* with Vs = 0 the mean stress -1/2 (txx + tzz) is the acoustic pressure and
  matches the closed-form 2D Green's function driven by -f'(t)
  (scaling and timing of the explosive source);
* in a homogeneous medium an explosive source radiates P waves only, so the
  recorded particle velocities do not depend on Vs (signs of the shear terms);
* the CPML absorbs (energy decays, no late growth);
* the stability limit vp dt / dx <= 1 / (sqrt(2) (9/8 + 1/24)) of the
  4th-order staggered scheme (stable just below it, blow-up just above);
* on the paper's three-layer model with a fluid top layer (Sec. 3.6.1) the
  energy, with the fluid's strain energy tau_xx^2 / (2 lambda), is still
  conserved exactly, the shear stress stays exactly zero wherever the
  harmonic shear average touches the fluid, and tau_xx = tau_zz in the fluid
  (no deviatoric stress without shear modulus).
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2604_14189_gb300 import inputs


def _mats(vp, vs, rho):
    """Mass and compliance of the staggered grid, as the engine defines them."""
    lam = rho * (vp ** 2 - 2 * vs ** 2)
    mu = rho * vs ** 2
    rx = np.concatenate([rho[:, 1:], rho[:, -1:]], axis=1)
    rz = np.concatenate([rho[1:, :], rho[-1:, :]], axis=0)
    mx = 0.5 * (rho + rx)  # 1 / buoyancy at vx points
    mz = 0.5 * (rho + rz)
    m01 = np.concatenate([mu[:, 1:], mu[:, -1:]], axis=1)
    m10 = np.concatenate([mu[1:, :], mu[-1:, :]], axis=0)
    m11 = np.concatenate([m10[:, 1:], m10[:, -1:]], axis=1)
    muxz = 4.0 / (1 / mu + 1 / m01 + 1 / m10 + 1 / m11)
    return lam, mu, mx, mz, muxz


def test_energy_conserved_without_pml():
    rng = np.random.default_rng(17)
    nz, nx, nt, dx, dt = 30, 36, 500, 5.0, 4e-4
    vp = rng.uniform(2000, 3000, (nz, nx))
    vs = vp / rng.uniform(1.6, 2.0, (nz, nx))
    rho = rng.uniform(1800, 2600, (nz, nx))
    w = np.zeros(nt)
    w[:40] = inputs.ricker(60.0, dt, 40, t0=0.008)
    p = oracle.make_problem(1, nz, nx, 0, dx, dt, nt, 1, 1, 30.0)
    _, wf = oracle.elastic_forward(p, np.stack([vp, vs, rho]), w[None],
                                   np.array([[15, 18]]), np.array([[[3, 3]]]),
                                   wavefield=True)
    f = wf[0]  # [nt+1][5][nz][nx]
    lam, mu, mx, mz, muxz = _mats(vp, vs, rho)
    l2m = lam + 2 * mu
    det = l2m ** 2 - lam ** 2
    E = []
    for k in range(45, nt):
        vx1, vz1 = f[k + 1, 0], f[k + 1, 1]   # v^{k+1/2}
        vx0, vz0 = f[k, 0], f[k, 1]           # v^{k-1/2}
        txx, tzz, txz = f[k, 2], f[k, 3], f[k, 4]  # tau^k
        kin = 0.5 * np.sum(mx * vx1 * vx0 + mz * vz1 * vz0)
        pot = 0.5 * np.sum((l2m * txx ** 2 - 2 * lam * txx * tzz + l2m * tzz ** 2) / det
                           + txz ** 2 / muxz)
        E.append(kin + pot)
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() / E[0] < 1e-11


@pytest.mark.parametrize("factor,stable", [(0.995, True), (1.01, False)])
def test_elastic_cfl_limit(factor, stable):
    """Von Neumann limit of the staggered 4th-order scheme in 2D: the P mode
    at the Nyquist wavenumber of both axes is the first to grow."""
    n, dx, vp = 30, 10.0, 2500.0
    limit = 1.0 / (np.sqrt(2.0) * (9.0 / 8.0 + 1.0 / 24.0))
    dt = factor * limit * dx / vp
    nt = 2000
    rng = np.random.default_rng(4)
    w = np.zeros(nt)
    w[:5] = rng.standard_normal(5)
    model = np.stack([np.full((n, n), vp), np.full((n, n), vp / 1.8), np.full((n, n), 2000.0)])
    p = oracle.make_problem(1, n, n, 0, dx, dt, nt, 1, 1, 10.0)
    with np.errstate(all="ignore"):
        d = oracle.elastic_forward(p, model, w[None], np.array([[15, 15]]),
                                   np.array([[[10, 12]]]))[0]
        early = np.abs(d[:, :, :50]).max()
        tail = d[:, :, -200:]
        late = np.abs(tail).max() if np.all(np.isfinite(tail)) else np.inf
    assert early > 0
    if stable:
        assert late < 10 * early
    else:
        assert late > 1e6 * early


def layered_model(ex, nz, nx):
    """The three-layer model of tests/golden/layered_example.json on an
    nz x nx grid, layers of equal thickness top to bottom: [3][nz][nx]."""
    z = np.arange(nz)[:, None] * 3 // nz + np.zeros((1, nx), dtype=int)
    return np.stack([np.asarray(ex[k])[z] for k in ("vp_m_s", "vs_m_s", "rho_kg_m3")])


def test_layered_example_fluid_top_energy_and_stress(golden):
    ex = golden("layered_example.json")
    assert ex["vs_m_s"][0] == 0.0 and min(ex["vs_m_s"][1:]) > 0
    nz, nx, dx, dt = 36, 40, 5.0, 4e-4
    model = layered_model(ex, nz, nx)
    vp, vs, rho = model
    f0 = ex["ricker_peak_hz"]
    nsrc = int(round(3.0 / f0 / dt))  # the wavelet over [0, 2 t0], then zero
    nt = nsrc + 150
    w = np.zeros(nt)
    w[:nsrc] = inputs.ricker(f0, dt, nsrc)
    p = oracle.make_problem(1, nz, nx, 0, dx, dt, nt, 1, 1, f0)
    # source in the middle (solid) layer: P and converted S waves meet the
    # fluid-solid interface
    _, wf = oracle.elastic_forward(p, model, w[None], np.array([[18, 20]]),
                                   np.array([[[3, 3]]]), wavefield=True)
    f = wf[0]  # [nt+1][5][nz][nx]
    with np.errstate(divide="ignore"):
        lam, mu, mx, mz, muxz = _mats(vp, vs, rho)
    fluid = mu == 0.0
    assert fluid.sum() == 12 * nx and np.all(fluid[:12])
    noshear = muxz == 0.0  # txz points touching a fluid cell (rows 0..11)
    assert np.all(noshear[:12]) and not noshear[12:].any()
    assert np.abs(f[:, 4][:, ~noshear]).max() > 0
    assert np.all(f[:, 4][:, noshear] == 0.0)
    assert np.abs(f[:, 2][:, fluid]).max() > 0
    assert np.array_equal(f[:, 2][:, fluid], f[:, 3][:, fluid])
    l2m = lam + 2 * mu
    solid = ~fluid
    det = (l2m ** 2 - lam ** 2)[solid]
    E = []
    for k in range(nsrc + 2, nt):
        vx1, vz1 = f[k + 1, 0], f[k + 1, 1]   # v^{k+1/2}
        vx0, vz0 = f[k, 0], f[k, 1]           # v^{k-1/2}
        txx, tzz, txz = f[k, 2], f[k, 3], f[k, 4]  # tau^k
        kin = 0.5 * np.sum(mx * vx1 * vx0 + mz * vz1 * vz0)
        ts, zs = txx[solid], tzz[solid]
        pot = 0.5 * (np.sum((l2m[solid] * ts ** 2 - 2 * lam[solid] * ts * zs
                             + l2m[solid] * zs ** 2) / det)
                     + np.sum(txx[fluid] ** 2 / lam[fluid])
                     + np.sum(txz[~noshear] ** 2 / muxz[~noshear]))
        E.append(kin + pot)
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() / E[0] < 1e-11


def _green_pressure(fdot, r, v, ts):
    """P(r,t) for P_tt = v^2 Lap P - f'(t) delta: the 2D Green's function with
    source term v^2 g, g = -f'/v^2."""
    out = np.zeros_like(ts)
    for k, t in enumerate(ts):
        if v * t > r:
            val, _ = integrate.quad(lambda s: fdot(t - (r / v) * np.cosh(s)), 0.0,
                                    np.arccosh(v * t / r), limit=200)
            out[k] = -val / (2 * np.pi * v ** 2)
    return out


def test_zero_shear_pressure_matches_green_function(golden):
    """The paper's acoustic example setting (Sec. 3.1.3, from
    tests/golden/acoustic_example.json) run through the elastic engine
    with Vs = 0; source at the centre, trace 200 m away."""
    ex = golden("acoustic_example.json")
    f0, v, dx, T = ex["ricker_peak_hz"], ex["vp_m_s"], 5.0, 0.2
    n = 161
    dt = 2.5e-4
    nt = int(round(T / dt))
    vp = np.full((n, n), v)
    model = np.stack([vp, 0 * vp, np.full((n, n), ex["rho_kg_m3"])])
    p = oracle.make_problem(1, n, n, 0, dx, dt, nt, 1, 1, f0)
    # the stress update from n to n+1 is centred at (n + 1/2) dt
    w = inputs.ricker(f0, dt, nt, shift=0.5)
    _, wf = oracle.elastic_forward(p, model, w[None], np.array([[80, 80]]),
                                   np.array([[[80, 120]]]), wavefield=True)
    P = -0.5 * (wf[0, 1:, 2, 80, 120] + wf[0, 1:, 3, 80, 120])  # at t = (k+1) dt
    ts = (np.arange(nt) + 1) * dt
    t0 = 1.5 / f0

    def rdot(t):
        a = (np.pi * f0 * (t - t0)) ** 2
        return np.exp(-a) * (-6 * np.pi ** 2 * f0 ** 2 * (t - t0) + 4 * np.pi ** 4
                             * f0 ** 4 * (t - t0) ** 3)

    a = _green_pressure(rdot, 40 * dx, v, ts)
    err = np.linalg.norm(P - a) / np.linalg.norm(a)
    assert err < 1.5e-2, err


def test_explosive_source_traces_independent_of_vs():
    f0, v, dx, dt, nt = 15.0, 2500.0, 5.0, 4e-4, 450
    n = 120
    out = []
    for vs in (0.0, v / 1.73):
        model = np.stack([np.full((n, n), v), np.full((n, n), vs), np.full((n, n), 2000.0)])
        p = oracle.make_problem(1, n, n, 20, dx, dt, nt, 1, 3, f0)
        d = oracle.elastic_forward(p, model, inputs.ricker(f0, dt, nt)[None],
                                   np.array([[60, 60]]),
                                   np.array([[[60, 100], [20, 60], [90, 90]]]))
        out.append(d[0])
    a, b = out
    assert np.abs(a).max() > 0
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 3e-2


def test_elastic_cpml_absorbs():
    nz = nx = 50
    dx, dt, nt = 5.0, 4e-4, 2500
    vp = np.full((nz, nx), 2500.0)
    model = np.stack([vp, vp / 1.73, np.full((nz, nx), 2000.0)])
    w = np.zeros(nt)
    w[:200] = inputs.ricker(30.0, dt, 200)
    p = oracle.make_problem(1, nz, nx, 20, dx, dt, nt, 1, 1, 30.0)
    _, wf = oracle.elastic_forward(p, model, w[None], np.array([[25, 25]]),
                                   np.array([[[0, 0]]]), wavefield=True)
    e = np.array([np.sum(x[:2] ** 2) for x in wf[0]])
    assert np.all(np.isfinite(e))
    assert e[-1] < 1e-4 * e.max()
    assert e[-1] < e[nt // 2]


# ---------------------------------------------------------------- reverse mode
def _small_elastic(seed=5, nt=160):
    rng = np.random.default_rng(seed)
    nz, nx, pml, dx, dt = 18, 22, 6, 5.0, 4e-4
    vp = 2500 + 100 * rng.standard_normal((nz, nx))
    vs = vp / 1.8
    rho = 2000 + 100 * rng.random((nz, nx))
    src = np.array([[3, 8], [4, 14]])
    rec = np.array([[[2, j] for j in range(2, 20, 3)]] * 2)
    p = oracle.make_problem(1, nz, nx, pml, dx, dt, nt, 2, rec.shape[1], 30.0, v_pml=3200.0)
    w = np.stack([inputs.ricker(40.0, dt, nt)] * 2) * 1e6
    return p, np.stack([vp, vs, rho]), w, src, rec, rng


def test_elastic_adjoint_dot_product():
    """<F w, d> = <w, F^T d> for the linear map wavelet -> traces (the
    adjoint is the exact transpose of the discrete recurrence)."""
    p, m, w, src, rec, rng = _small_elastic()
    d = oracle.elastic_forward(p, m, w, src, rec)
    db = rng.standard_normal(d.shape)
    wg = oracle.elastic_adjoint(p, m, db, src, rec)
    lhs, rhs = np.sum(d * db), np.sum(w * wg)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_elastic_adjoint_of_a_single_trace_sample():
    """Brute force on one entry: the adjoint of a unit impulse in one trace
    sample equals the column of the forward map (the response of that sample
    to a unit wavelet sample), checked for a few wavelet samples."""
    p, m, w, src, rec, rng = _small_elastic(nt=40)
    db = np.zeros((p.nshot, 2, p.nrec, p.nt))
    db[1, 1, 3, 30] = 1.0
    wg = oracle.elastic_adjoint(p, m, db, src, rec)
    for n in (0, 7, 19):
        e = np.zeros_like(w)
        e[1, n] = 1.0
        d = oracle.elastic_forward(p, m, e, src, rec)
        assert abs(d[1, 1, 3, 30] - wg[1, n]) <= 1e-12 * max(abs(d[1, 1, 3, 30]), 1e-30)


def _taper(a):
    a = a.copy()
    a[:2] = 0
    a[-2:] = 0
    a[:, :2] = 0
    a[:, -2:] = 0
    return a


def test_elastic_gradient_matches_finite_differences():
    """Central differences of the misfit along smooth perturbations of vp,
    vs and rho (zero on the interior edge, so the edge-replicated padding is
    unchanged) against <grad, dm>; fixes the chain rule through Hooke's
    parameters, the buoyancy averages and the harmonic shear average."""
    from scipy.ndimage import gaussian_filter

    p, m, w, src, rec, rng = _small_elastic()
    mt = m.copy()
    mt[0, 8:12, 8:14] *= 1.05
    mt[1, 5:9, 10:16] *= 0.95
    mt[2, 10:14, 4:9] *= 1.04
    dobs = oracle.elastic_forward(p, mt, w, src, rec)
    g, J = oracle.elastic_gradient(p, m, w, src, rec, dobs)
    d = oracle.elastic_forward(p, m, w, src, rec)
    assert abs(J - 0.5 * np.sum((d - dobs) ** 2)) <= 1e-12 * J
    for k in range(3):
        dm = np.zeros_like(m)
        dm[k] = _taper(gaussian_filter(rng.standard_normal(m[k].shape), 2.0)) * m[k].mean() * 1e-3
        h = 0.5
        Jp = 0.5 * np.sum((oracle.elastic_forward(p, m + h * dm, w, src, rec) - dobs) ** 2)
        Jm = 0.5 * np.sum((oracle.elastic_forward(p, m - h * dm, w, src, rec) - dobs) ** 2)
        fd = (Jp - Jm) / (2 * h)
        an = np.sum(g[k] * dm[k])
        assert abs(fd - an) <= 2e-5 * abs(fd), (k, fd, an)
