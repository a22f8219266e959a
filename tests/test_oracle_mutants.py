"""The oracle's pins catch plausible mistakes in the oracle itself.

Each case plants one mistake in a scratch copy of the C oracle: a wrong
coefficient, sign, index or stagger, a dropped term, or a transposed operand.
The case builds the copy and runs the pins that should notice the mistake,
with the copy standing in for the oracle, and at least one of them must fail.
An unmodified copy must pass the same pins, so the harness itself is checked
too.  CPU only; the scratch copies live under _build/ (not versioned).
"""
import importlib.util
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRATCH = os.path.join(ROOT, "_build", "oracle_mutants")
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import test_oracle_acoustic as TA  # noqa: E402
import test_oracle_elastic as TE  # noqa: E402

A, E = "acoustic", "elastic"
# pins: (module, test function, arguments)
STENCIL2 = (A, "test_stencil_exact_on_polynomials", dict(kind=0, order=2))
STENCIL1 = (A, "test_stencil_exact_on_polynomials", dict(kind=1, order=1))
NYQUIST = (A, "test_nyquist_symbol_and_cfl_bound", {})
GREEN = (A, "test_green_function_convergence", {})
ENERGY = (A, "test_energy_conserved_without_pml", {})
DECAY = (A, "test_energy_decays_with_cpml", {})
REFLECT = (A, "test_cpml_reflection_below_one_percent", {})
TRANSPOSE = (A, "test_adjoint_equals_dense_transpose", {})
REACH = (A, "test_adjoint_reaches_pml", {})
FD = (A, "test_gradient_matches_central_differences_all_cells", {})
E_ENERGY = (E, "test_energy_conserved_without_pml", {})
E_LAYERED = (E, "test_layered_example_fluid_top_energy_and_stress", {})
E_GREEN = (E, "test_zero_shear_pressure_matches_green_function", {})
E_VS = (E, "test_explosive_source_traces_independent_of_vs", {})
E_DOT = (E, "test_elastic_adjoint_dot_product", {})
E_ONE = (E, "test_elastic_adjoint_of_a_single_trace_sample", {})
E_FD = (E, "test_elastic_gradient_matches_finite_differences", {})

# (name, file, text, replacement, pins of which at least one must fail)
CASES = [
    ("c2_coefficient", "common.c", "8.0 / 315.0", "8.0 / 316.0", [STENCIL2, NYQUIST]),
    ("c1_sign", "common.c", "4.0 / 105.0", "-4.0 / 105.0", [STENCIL1]),
    ("laplacian_sign", "acoustic.c",
     "out->u[c] = 2.0 * in->u[c] - in->up[c] + g->K[c] * br;",
     "out->u[c] = 2.0 * in->u[c] - in->up[c] - g->K[c] * br;", [GREEN, ENERGY]),
    ("dropped_zeta_z", "acoustic.c", "const double br = Wx + zx + Wz + zz;",
     "const double br = Wx + zx + Wz;", [TRANSPOSE, DECAY, REFLECT]),
    ("records_u_n", "acoustic.c",
     "data[((size_t)s * p->nrec + r) * p->nt + n] = nxt->u[cr];",
     "data[((size_t)s * p->nrec + r) * p->nt + n] = cur->u[cr];", [GREEN, TRANSPOSE]),
    ("source_without_K", "acoustic.c",
     "nxt->u[cs] += g.K[cs] * wavelet[(size_t)s * p->nt + n];",
     "nxt->u[cs] += wavelet[(size_t)s * p->nt + n];", [GREEN, TRANSPOSE]),
    ("adjoint_u_prev_sign", "acoustic.c", "aout->up[c] += -lun;", "aout->up[c] += lun;",
     [TRANSPOSE]),
    ("adjoint_psi_sign", "acoustic.c", "acc(g, aout->psx, i, j - k, -ORC_C1[k] * wx);",
     "acc(g, aout->psx, i, j - k, ORC_C1[k] * wx);", [TRANSPOSE, REACH]),
    ("imaging_without_source", "acoustic.c", "full[cs] += f[n];", "", [FD]),
    ("dK_dv_factor", "acoustic.c",
     "grad[(size_t)i * nx + j] = sum * 2.0 * v * p->dt * p->dt / (p->dx * p->dx);",
     "grad[(size_t)i * nx + j] = sum * v * p->dt * p->dt / (p->dx * p->dx);", [FD]),
    ("cpml_b_sign", "common.c", "b[j] = sigma / (sigma + alpha) * (a[j] - 1.0);",
     "b[j] = sigma / (sigma + alpha) * (1.0 - a[j]);", [DECAY, REFLECT]),
    ("cpml_alpha_reversed", "common.c", "const double alpha = M_PI * f_ref * (1.0 - rho);",
     "const double alpha = M_PI * f_ref * rho;", [DECAY, REFLECT]),
    ("adjoint_zeta_a_for_b", "acoustic.c", "aout->zex[c] += g->ax[j] * tzx;",
     "aout->zex[c] += g->bx[j] * tzx;", [TRANSPOSE, REACH]),
    ("arithmetic_shear_mean", "elastic.c",
     ": 4.0 / (1.0 / m00 + 1.0 / m01 + 1.0 / m10 + 1.0 / m11);",
     ": 0.25 * (m00 + m01 + m10 + m11);", [E_ENERGY, E_LAYERED]),
    # a harmonic mean regularised against zero moduli: shear leaks into the fluid
    ("shear_mean_regularised", "elastic.c",
     "g->muxz[c] = (m00 == 0.0 || m01 == 0.0 || m10 == 0.0 || m11 == 0.0)\n"
     "                       ? 0.0\n"
     "                       : 4.0 / (1.0 / m00 + 1.0 / m01 + 1.0 / m10 + 1.0 / m11);",
     "g->muxz[c] = 4.0 / (1.0 / (m00 + 1e-6) + 1.0 / (m01 + 1e-6) + 1.0 / (m10 + 1e-6)"
     " + 1.0 / (m11 + 1e-6));", [E_LAYERED]),
    ("lambda_plus_mu", "elastic.c",
     "const double l2m = g.lam[c] + 2.0 * g.mu[c];\n          txx[c]",
     "const double l2m = g.lam[c] + 1.0 * g.mu[c];\n          txx[c]", [E_ENERGY, E_LAYERED]),
    ("harmonic_x_buoyancy", "elastic.c",
     "g->bux[c] = 2.0 / (rho[c] + rho[(size_t)i * NX + j1]);",
     "g->bux[c] = 0.5 * (1.0 / rho[c] + 1.0 / rho[(size_t)i * NX + j1]);", [E_ENERGY]),
    ("source_into_txx_only", "elastic.c", "      tzz[cs] += amp;\n", "", [E_GREEN, E_VS]),
    ("vx_shear_stagger", "elastic.c",
     "const double dzt = dmz(&g, txz, i, j) * idx; /* at (i, j+1/2) */",
     "const double dzt = dpz(&g, txz, i, j) * idx; /* at (i, j+1/2) */", [E_ENERGY, E_VS]),
    ("p1_integer_point_profile", "elastic.c",
     "p1[c] = g.axh[j] * p1[c] + g.bxh[j] * dxt;",
     "p1[c] = g.ax[j] * p1[c] + g.bx[j] * dxt;", [E_DOT, E_ONE]),
    ("txz_without_dt", "elastic.c",
     "txz[c] += dt * g.muxz[c] * (ezx + p7[c] + exz + p8[c]);",
     "txz[c] += g.muxz[c] * (ezx + p7[c] + exz + p8[c]);", [E_ENERGY, E_VS]),
    ("adjoint_hooke_transposed", "elastic.c",
     "const double Ex = dt * (l2m * atxx[c] + g->lam[c] * atzz[c]);",
     "const double Ex = dt * (g->lam[c] * atxx[c] + l2m * atzz[c]);", [E_DOT, E_ONE]),
    ("dlambda_dvs_sign", "elastic.c", "gvs[c] = glam[c] * (-4.0 * rho[c] * vs[c])",
     "gvs[c] = glam[c] * (4.0 * rho[c] * vs[c])", [E_FD]),
    ("dmu_factor", "elastic.c", "gmu[c] += 2.0 * dt * (atxx[c] * ex[c] + atzz[c] * ez[c]);",
     "gmu[c] += 1.0 * dt * (atxx[c] * ex[c] + atzz[c] * ez[c]);", [E_FD]),
]


def _copy(tag, patch=None):
    """A built scratch copy of the oracle package, with `patch` applied."""
    top = os.path.join(SCRATCH, tag)
    if os.path.exists(top):
        shutil.rmtree(top)
    d = os.path.join(top, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), d,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    if patch:
        fname, old, new = patch
        path = os.path.join(d, fname)
        src = open(path).read()
        assert src.count(old) == 1, (tag, old)
        with open(path, "w") as f:
            f.write(src.replace(old, new))
    name = "oracle_copy_" + tag
    spec = importlib.util.spec_from_file_location(name, os.path.join(d, "__init__.py"),
                                                  submodule_search_locations=[d])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def _run(copy, pin, golden, quiet=False):
    """Run one pin with `copy` in place of the oracle (quiet: no warnings for
    the overflow of a mutant that blows up)."""
    module, fn, kwargs = pin
    T = TA if module == A else TE
    f = getattr(T, fn)
    args = f.__code__.co_varnames[:f.__code__.co_argcount]
    kw = dict(kwargs, golden=golden) if "golden" in args else dict(kwargs)
    with pytest.MonkeyPatch.context() as mp, np.errstate(all="ignore" if quiet else "warn"):
        mp.setattr(T, "oracle", copy)
        f(**kw)


def test_unmodified_copy_passes_every_pin(golden):
    copy = _copy("unmodified")
    pins = []
    for case in CASES:
        for pin in case[4]:
            if pin not in pins:
                pins.append(pin)
    for pin in pins:
        _run(copy, pin, golden)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(case, golden):
    name, fname, old, new, pins = case
    copy = _copy(name, (fname, old, new))
    failed = []
    for pin in pins:
        try:
            _run(copy, pin, golden, quiet=True)
        except AssertionError:
            failed.append(pin[1])
    assert failed, f"{name}: no pin failed among {[p[1] for p in pins]}"
