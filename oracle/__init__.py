"""FP64 CPU oracle for the SWEEP finite-difference wave solvers.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_2604_14189_gb300``) never imports it and shares no code with it.

The numerics live in plain C (``acoustic.c``, ``elastic.c``, ``common.c``),
compiled here with gcc (no fast-math) into ``liboracle.so`` on first use; this
module only marshals numpy arrays through ctypes.  What each routine computes,
and the readings of the paper it follows, are stated in ``oracle.h``.  The
learned gradient preconditioner's network (U-Net forward, backward, MSE loss,
Adam) is plain numpy in FP64: ``oracle/unet.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["common.c", "acoustic.c", "elastic.c"]
_HDRS = ["oracle.h", "oracle_internal.h"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ACOUSTIC = 0
ELASTIC = 1
F_PADDED_MODEL = 0x1
F_RESIDUAL_IN = 0x2


class Problem(ctypes.Structure):
    _fields_ = [
        ("physics", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("pml", ctypes.c_int32),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("nt", ctypes.c_int32),
        ("nshot", ctypes.c_int32),
        ("nrec", ctypes.c_int32),
        ("f_ref", ctypes.c_double),
        ("v_pml", ctypes.c_double),
        ("flags", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its sources."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDRS]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= lib_m for d in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER(Problem)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_stencil_1d.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            lib.oracle_stencil_1d.restype = None
            lib.oracle_cpml_profile.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
            lib.oracle_cpml_profile.restype = None
            for name in ("oracle_acoustic_forward", "oracle_elastic_forward"):
                f = getattr(lib, name)
                f.argtypes = [P, dp, dp, ip, ip, dp, dp]
                f.restype = ctypes.c_int
            lib.oracle_acoustic_adjoint.argtypes = [P, dp, dp, ip, ip, dp]
            lib.oracle_acoustic_adjoint.restype = ctypes.c_int
            lib.oracle_acoustic_gradient.argtypes = [P, dp, dp, ip, ip, dp, dp, dp]
            lib.oracle_elastic_adjoint.argtypes = [P, dp, dp, ip, ip, dp]
            lib.oracle_elastic_gradient.argtypes = [P, dp, dp, ip, ip, dp, dp, dp]
            lib.oracle_acoustic_gradient.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def make_problem(physics, nz, nx, pml, dx, dt, nt, nshot, nrec, f_ref, flags=0,
                 v_pml=0.0):
    return Problem(physics, nz, nx, pml, float(dx), float(dt), nt, nshot, nrec,
                   float(f_ref), float(v_pml), flags)


def set_threads(n: int | None) -> None:
    """Set the OpenMP thread count used by later oracle calls."""
    lib = _load()
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(int(n if n else os.cpu_count()))
    except OSError:
        pass
    del lib


def stencil_1d(kind: int, f) -> np.ndarray:
    lib = _load()
    f = _d(f)
    out = np.empty_like(f)
    lib.oracle_stencil_1d(kind, f.size, _ptr(f, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def cpml_profile(n_int, pml, dx, dt, vmax, f_ref, half=False):
    lib = _load()
    a = np.zeros(n_int + 2 * pml)
    b = np.zeros(n_int + 2 * pml)
    lib.oracle_cpml_profile(n_int, pml, dx, dt, vmax, f_ref, int(half),
                            _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double))
    return a, b


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")


def acoustic_forward(p: Problem, model, wavelet, src, rec, wavefield=False):
    """Returns data [nshot][nrec][nt] (and u^0..u^nt per shot if wavefield)."""
    lib = _load()
    model, wavelet, src, rec = _d(model), _d(wavelet), _i(src), _i(rec)
    data = np.zeros((p.nshot, p.nrec, p.nt))
    NZ, NX = p.nz + 2 * p.pml, p.nx + 2 * p.pml
    wf = np.zeros((p.nshot, p.nt + 1, NZ, NX)) if wavefield else None
    rc = lib.oracle_acoustic_forward(
        ctypes.byref(p), _ptr(model, ctypes.c_double), _ptr(wavelet, ctypes.c_double),
        _ptr(src, ctypes.c_int32), _ptr(rec, ctypes.c_int32),
        _ptr(data, ctypes.c_double),
        _ptr(wf, ctypes.c_double) if wf is not None else None)
    _check(rc)
    return (data, wf) if wavefield else data


def acoustic_adjoint(p: Problem, model, adj_data, src, rec):
    lib = _load()
    model, adj_data, src, rec = _d(model), _d(adj_data), _i(src), _i(rec)
    out = np.zeros((p.nshot, p.nt))
    rc = lib.oracle_acoustic_adjoint(
        ctypes.byref(p), _ptr(model, ctypes.c_double), _ptr(adj_data, ctypes.c_double),
        _ptr(src, ctypes.c_int32), _ptr(rec, ctypes.c_int32), _ptr(out, ctypes.c_double))
    _check(rc)
    return out


def acoustic_gradient(p: Problem, model, wavelet, src, rec, d_obs):
    """Returns (grad [nz][nx], misfit)."""
    lib = _load()
    model, wavelet, src, rec, d_obs = _d(model), _d(wavelet), _i(src), _i(rec), _d(d_obs)
    grad = np.zeros((p.nz, p.nx))
    J = ctypes.c_double(0.0)
    rc = lib.oracle_acoustic_gradient(
        ctypes.byref(p), _ptr(model, ctypes.c_double), _ptr(wavelet, ctypes.c_double),
        _ptr(src, ctypes.c_int32), _ptr(rec, ctypes.c_int32), _ptr(d_obs, ctypes.c_double),
        _ptr(grad, ctypes.c_double), ctypes.byref(J))
    _check(rc)
    return grad, J.value


def elastic_forward(p: Problem, model, wavelet, src, rec, wavefield=False):
    """Returns data [nshot][2][nrec][nt] (and fields per step if wavefield)."""
    lib = _load()
    model, wavelet, src, rec = _d(model), _d(wavelet), _i(src), _i(rec)
    data = np.zeros((p.nshot, 2, p.nrec, p.nt))
    NZ, NX = p.nz + 2 * p.pml, p.nx + 2 * p.pml
    wf = np.zeros((p.nshot, p.nt + 1, 5, NZ, NX)) if wavefield else None
    rc = lib.oracle_elastic_forward(
        ctypes.byref(p), _ptr(model, ctypes.c_double), _ptr(wavelet, ctypes.c_double),
        _ptr(src, ctypes.c_int32), _ptr(rec, ctypes.c_int32),
        _ptr(data, ctypes.c_double),
        _ptr(wf, ctypes.c_double) if wf is not None else None)
    _check(rc)
    return (data, wf) if wavefield else data


def elastic_adjoint(p: Problem, model, adj_data, src, rec):
    """Wavelet adjoint [nshot][nt] of the elastic data map for adj_data
    [nshot][2][nrec][nt]."""
    lib = _load()
    model, adj_data, src, rec = _d(model), _d(adj_data), _i(src), _i(rec)
    wg = np.zeros((p.nshot, p.nt))
    rc = lib.oracle_elastic_adjoint(
        ctypes.byref(p), _ptr(model, ctypes.c_double), _ptr(adj_data, ctypes.c_double),
        _ptr(src, ctypes.c_int32), _ptr(rec, ctypes.c_int32), _ptr(wg, ctypes.c_double))
    _check(rc)
    return wg


def elastic_gradient(p: Problem, model, wavelet, src, rec, d_obs):
    """(grad [3][nz][nx] of the misfit w.r.t. (vp, vs, rho), misfit J)."""
    lib = _load()
    model, wavelet, src, rec, d_obs = _d(model), _d(wavelet), _i(src), _i(rec), _d(d_obs)
    grad = np.zeros((3, p.nz, p.nx))
    J = ctypes.c_double(0.0)
    rc = lib.oracle_elastic_gradient(
        ctypes.byref(p), _ptr(model, ctypes.c_double), _ptr(wavelet, ctypes.c_double),
        _ptr(src, ctypes.c_int32), _ptr(rec, ctypes.c_int32), _ptr(d_obs, ctypes.c_double),
        _ptr(grad, ctypes.c_double), ctypes.byref(J))
    _check(rc)
    return grad, J.value
