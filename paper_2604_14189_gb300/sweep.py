"""Thin ctypes binding of the C ABI in ``include/sweep.h`` (``libsweep.so``).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Tensors must be CUDA tensors (float32 / int32, contiguous);
PyTorch supplies device memory and the current stream.  There is no CPU
fallback: importing this module fails if the library cannot be loaded.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading

import torch

from . import build as _build

ACOUSTIC = 0
ELASTIC = 1
MODE_FORWARD = 0
MODE_ADJOINT = 1
MODE_GRADIENT = 2
F_PADDED_MODEL = 0x1
F_RESIDUAL_IN = 0x2
F_ROWS16 = 0x4
F_ONE_LAUNCH = 0x8
F_DETERMINISTIC = 0x10

OK = 0
EINVAL, ECFL, EBOUNDS, EWORKSPACE, ECUDA, ETIMEOUT, ENONFINITE, EMODEL, EUNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7, -8, -9)
ETOOBIG = -10
DOT_NOALLOC_MAX_N = 33554432

# Every symbol declared in include/sweep.h.
EXPORTS = ("sweep_workspace_bytes", "sweep_forward", "sweep_adjoint", "sweep_gradient",
           "sweep_dot_workspace_bytes", "sweep_dot", "sweep_status", "sweep_strerror",
           "sweep_kernel_launches", "sweep_profile_enable", "sweep_profile_read",
           "sweep_dot_noalloc", "sweep_capture_begin", "sweep_capture_end",
           "sweep_graph_launch", "sweep_graph_kernels", "sweep_graph_destroy",
           "sweep_check_wait_timeout", "sweep_check_barrier_timeout", "sweep_gradient_batch",
           "sweep_forward_batch")
K_AC_FWD, K_AC_BWD, K_EL_VEL, K_EL_STR = 0, 1, 2, 3
K_AC_FWD_LOOP, K_AC_BWD_LOOP = 8, 9
K_EL_ADJ = 10  # elastic transposed step


class Problem(ctypes.Structure):
    """Mirror of ``sweep_problem``."""
    _fields_ = [
        ("physics", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("pml", ctypes.c_int32),
        ("dx", ctypes.c_float),
        ("dt", ctypes.c_float),
        ("nt", ctypes.c_int32),
        ("nshot", ctypes.c_int32),
        ("nrec", ctypes.c_int32),
        ("f_ref", ctypes.c_float),
        ("v_pml", ctypes.c_float),
        ("flags", ctypes.c_int32),
    ]

    def __repr__(self):
        return "Problem(" + ", ".join(f"{n}={getattr(self, n)}" for n, _ in self._fields_) + ")"


def problem(physics=ACOUSTIC, *, nz, nx, pml, dx, dt, nt, nshot, nrec, f_ref=10.0,
            v_pml=0.0, flags=0) -> Problem:
    return Problem(physics, nz, nx, pml, dx, dt, nt, nshot, nrec, f_ref, v_pml, flags)


class SweepError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libsweep.so (building it first if missing)."""
    path = path or _build.LIB
    if not os.path.exists(path):
        _build.build()
    lib = ctypes.CDLL(path)
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    P = ctypes.POINTER(Problem)
    lib.sweep_workspace_bytes.argtypes = [P, i32]
    lib.sweep_workspace_bytes.restype = sz
    lib.sweep_forward.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sweep_forward.restype = i32
    lib.sweep_adjoint.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sweep_adjoint.restype = i32
    lib.sweep_gradient.argtypes = [P, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sweep_gradient.restype = i32
    lib.sweep_dot_workspace_bytes.argtypes = []
    lib.sweep_dot_workspace_bytes.restype = sz
    lib.sweep_dot.argtypes = [vp, vp, ctypes.c_int64, vp, vp, sz, vp]
    lib.sweep_dot.restype = i32
    lib.sweep_dot_noalloc.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    lib.sweep_dot_noalloc.restype = i32
    lib.sweep_status.argtypes = [vp, vp]
    lib.sweep_status.restype = i32
    lib.sweep_strerror.argtypes = [i32]
    lib.sweep_strerror.restype = ctypes.c_char_p
    lib.sweep_kernel_launches.argtypes = []
    lib.sweep_kernel_launches.restype = ctypes.c_ulonglong
    lib.sweep_profile_enable.argtypes = [i32]
    lib.sweep_profile_enable.restype = i32
    lib.sweep_profile_read.argtypes = [i32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]
    lib.sweep_profile_read.restype = i32
    lib.sweep_capture_begin.argtypes = [vp]
    lib.sweep_capture_begin.restype = i32
    lib.sweep_capture_end.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p)]
    lib.sweep_capture_end.restype = i32
    lib.sweep_graph_launch.argtypes = [vp, vp]
    lib.sweep_graph_launch.restype = i32
    lib.sweep_graph_kernels.argtypes = [vp]
    lib.sweep_graph_kernels.restype = i32
    lib.sweep_graph_destroy.argtypes = [vp]
    lib.sweep_graph_destroy.restype = None
    lib.sweep_check_wait_timeout.argtypes = [vp, sz, vp]
    lib.sweep_check_wait_timeout.restype = i32
    lib.sweep_check_barrier_timeout.argtypes = [vp, sz, vp]
    lib.sweep_check_barrier_timeout.restype = i32
    lib.sweep_gradient_batch.argtypes = [i32] + [vp] * 11
    lib.sweep_gradient_batch.restype = i32
    lib.sweep_forward_batch.argtypes = [i32] + [vp] * 9
    lib.sweep_forward_batch.restype = i32
    return lib


_lib = load_library()


def lib() -> ctypes.CDLL:
    return _lib


def strerror(code: int) -> str:
    return _lib.sweep_strerror(int(code)).decode()


def kernel_launches() -> int:
    return int(_lib.sweep_kernel_launches())


def profile_enable(on) -> None:
    """True: record every kernel class; an int: bit mask of classes (1 << K_*);
    False / 0: stop recording."""
    mask = -1 if on is True else (0 if on is False else int(on))
    _lib.sweep_profile_enable(mask)


def profile_read(kernel: int) -> tuple[float, int]:
    """(summed device ms, launches) of a kernel class since profile_enable(True)."""
    ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
    rc = _lib.sweep_profile_read(kernel, ctypes.byref(ms), ctypes.byref(n))
    if rc != OK:
        raise SweepError(rc, "sweep_profile_read")
    return ms.value, n.value


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("sweep: tensors must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("sweep: tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check_dtype(t, dt, name):
    if t is not None and t.dtype != dt:
        raise TypeError(f"sweep: {name} must be {dt}, got {t.dtype}")


def _check_size(t, shape, name):
    """The C ABI sees only pointers, so a tensor with fewer elements than the
    call touches would be read or written out of bounds on the GPU: the
    element count must be that of `shape` (any view of the same layout)."""
    if t is None:
        return
    n = 1
    for d in shape:
        n *= int(d)
    if t.numel() != n:
        raise ValueError(f"sweep: {name} must hold {n} elements {tuple(shape)}, "
                         f"got shape {tuple(t.shape)}")


def _model_shape(p: Problem):
    npar = 3 if p.physics == ELASTIC else 1
    if p.flags & F_PADDED_MODEL:
        nz, nx = p.nz + 2 * p.pml, p.nx + 2 * p.pml
    else:
        nz, nx = p.nz, p.nx
    return (npar, nz, nx)


def _check_inputs(p: Problem, model, wavelet=None, src=None, rec=None):
    _check_size(model, _model_shape(p), "model")
    _check_size(wavelet, (p.nshot, p.nt), "wavelet")
    _check_size(src, (p.nshot, 2), "src")
    _check_size(rec, (p.nshot, p.nrec, 2), "rec")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_bytes(p: Problem, mode: int) -> int:
    n = int(_lib.sweep_workspace_bytes(ctypes.byref(p), mode))
    if n == 0:
        raise SweepError(EINVAL, "sweep_workspace_bytes")
    return n


def alloc_workspace(p: Problem, mode: int, device=None) -> torch.Tensor:
    """A uint8 CUDA tensor big enough (and 256-byte aligned) for `mode`."""
    n = workspace_bytes(p, mode)
    ws = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-ws.data_ptr()) % 256
    return ws[off:off + n]


def _ws_args(ws):
    return ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def check_wait_timeout(ws: torch.Tensor, stream=None) -> None:
    """Runs the timeout diagnostic on `ws` (see sweep_check_wait_timeout)."""
    w, wn = _ws_args(ws)
    rc = _lib.sweep_check_wait_timeout(w, wn, _stream(stream))
    if rc != OK:
        raise SweepError(rc, "sweep_check_wait_timeout")


def check_barrier_timeout(ws: torch.Tensor, stream=None) -> None:
    """Runs the grid-barrier timeout diagnostic on `ws` (see
    sweep_check_barrier_timeout)."""
    w, wn = _ws_args(ws)
    rc = _lib.sweep_check_barrier_timeout(w, wn, _stream(stream))
    if rc != OK:
        raise SweepError(rc, "sweep_check_barrier_timeout")


def status(ws: torch.Tensor, stream=None) -> int:
    return int(_lib.sweep_status(ctypes.c_void_p(ws.data_ptr()), _stream(stream)))


def _finish(rc, ws, where, stream, sync):
    if rc != OK:
        raise SweepError(rc, where)
    if sync and not getattr(_capture_state, "on", False):
        st = status(ws, stream)
        if st != OK:
            raise SweepError(st, where)


def sweep_forward(p: Problem, model, wavelet, src, rec, data=None, ws=None, stream=None,
                  sync=True):
    """data [nshot][ncomp][nrec][nt] (float32, CUDA)."""
    _check_dtype(model, torch.float32, "model")
    _check_dtype(wavelet, torch.float32, "wavelet")
    _check_dtype(src, torch.int32, "src")
    _check_dtype(rec, torch.int32, "rec")
    ncomp = 2 if p.physics == ELASTIC else 1
    _check_inputs(p, model, wavelet, src, rec)
    if data is None:
        data = torch.empty((p.nshot, ncomp, p.nrec, p.nt), dtype=torch.float32,
                           device=model.device)
    _check_dtype(data, torch.float32, "data")
    _check_size(data, (p.nshot, ncomp, p.nrec, p.nt), "data")
    if ws is None:
        ws = alloc_workspace(p, MODE_FORWARD, model.device)
    w, wn = _ws_args(ws)
    rc = _lib.sweep_forward(ctypes.byref(p), _ptr(model), _ptr(wavelet), _ptr(src), _ptr(rec),
                            _ptr(data), w, wn, _stream(stream))
    _finish(rc, ws, "sweep_forward", stream, sync)
    return data


def sweep_adjoint(p: Problem, model, adj_data, src, rec, wavelet_grad=None, ws=None,
                  stream=None, sync=True):
    """wavelet_grad [nshot][nt]."""
    _check_dtype(model, torch.float32, "model")
    _check_dtype(adj_data, torch.float32, "adj_data")
    _check_dtype(src, torch.int32, "src")
    _check_dtype(rec, torch.int32, "rec")
    ncomp = 2 if p.physics == ELASTIC else 1
    _check_inputs(p, model, None, src, rec)
    _check_size(adj_data, (p.nshot, ncomp, p.nrec, p.nt), "adj_data")
    if wavelet_grad is None:
        wavelet_grad = torch.empty((p.nshot, p.nt), dtype=torch.float32, device=model.device)
    _check_dtype(wavelet_grad, torch.float32, "wavelet_grad")
    _check_size(wavelet_grad, (p.nshot, p.nt), "wavelet_grad")
    if ws is None:
        ws = alloc_workspace(p, MODE_ADJOINT, model.device)
    w, wn = _ws_args(ws)
    rc = _lib.sweep_adjoint(ctypes.byref(p), _ptr(model), _ptr(adj_data), _ptr(src), _ptr(rec),
                            _ptr(wavelet_grad), w, wn, _stream(stream))
    _finish(rc, ws, "sweep_adjoint", stream, sync)
    return wavelet_grad


def sweep_gradient(p: Problem, model, wavelet, src, rec, d_obs, grad=None, misfit=None,
                   illum=None, want_illum=False, ws=None, stream=None, sync=True):
    """Returns (grad, misfit (device float64 scalar), illum or None); grad is
    [nz][nx] (acoustic: d J / d vp) or [3][nz][nx] (elastic: vp, vs, rho)."""
    _check_dtype(model, torch.float32, "model")
    _check_dtype(wavelet, torch.float32, "wavelet")
    _check_dtype(src, torch.int32, "src")
    _check_dtype(rec, torch.int32, "rec")
    _check_dtype(d_obs, torch.float32, "d_obs")
    ncomp = 2 if p.physics == ELASTIC else 1
    _check_inputs(p, model, wavelet, src, rec)
    _check_size(d_obs, (p.nshot, ncomp, p.nrec, p.nt), "d_obs")
    dev = model.device
    shape = (3, p.nz, p.nx) if p.physics == ELASTIC else (p.nz, p.nx)
    if grad is None:
        grad = torch.empty(shape, dtype=torch.float32, device=dev)
    if misfit is None:
        misfit = torch.empty((), dtype=torch.float64, device=dev)
    if illum is None and want_illum:
        illum = torch.empty((p.nz, p.nx), dtype=torch.float32, device=dev)
    _check_dtype(grad, torch.float32, "grad")
    _check_size(grad, shape, "grad")
    _check_dtype(misfit, torch.float64, "misfit")
    if misfit.numel() != 1:
        raise ValueError("sweep: misfit must be a one-element float64 tensor")
    _check_dtype(illum, torch.float32, "illum")
    _check_size(illum, (p.nz, p.nx), "illum")
    if ws is None:
        ws = alloc_workspace(p, MODE_GRADIENT, dev)
    w, wn = _ws_args(ws)
    rc = _lib.sweep_gradient(ctypes.byref(p), _ptr(model), _ptr(wavelet), _ptr(src), _ptr(rec),
                             _ptr(d_obs), _ptr(grad), _ptr(misfit), _ptr(illum), w, wn,
                             _stream(stream))
    _finish(rc, ws, "sweep_gradient", stream, sync)
    return grad, misfit, illum


def sweep_gradient_batch(problems, models, wavelets, srcs, recs, d_obs, grads=None,
                         misfits=None, ws=None, stream=None, sync=True):
    """Acoustic gradients of several problems in one call (sweep_gradient_batch):
    lists with one entry per problem; returns (grads, misfits).  Each problem
    gets its own workspace (allocated here when ``ws`` is None)."""
    n = len(problems)
    if not (len(models) == len(wavelets) == len(srcs) == len(recs) == len(d_obs) == n):
        raise ValueError("sweep_gradient_batch: one entry per problem in every list")
    if n == 0:
        return [], []
    dev = models[0].device
    grads = list(grads) if grads is not None else [
        torch.empty((p.nz, p.nx), dtype=torch.float32, device=dev) for p in problems]
    misfits = list(misfits) if misfits is not None else [
        torch.empty((), dtype=torch.float64, device=dev) for _ in problems]
    ws = list(ws) if ws is not None else [
        alloc_workspace(p, MODE_GRADIENT, dev) for p in problems]
    for i, p in enumerate(problems):
        if p.physics != ACOUSTIC:
            raise SweepError(EUNSUPPORTED, "sweep_gradient_batch")
        for t, dt, name in ((models[i], torch.float32, "model"),
                            (wavelets[i], torch.float32, "wavelet"),
                            (srcs[i], torch.int32, "src"), (recs[i], torch.int32, "rec"),
                            (d_obs[i], torch.float32, "d_obs"), (grads[i], torch.float32, "grad"),
                            (misfits[i], torch.float64, "misfit")):
            _check_dtype(t, dt, f"{name}[{i}]")
        _check_inputs(p, models[i], wavelets[i], srcs[i], recs[i])
        _check_size(d_obs[i], (p.nshot, 1, p.nrec, p.nt), f"d_obs[{i}]")
        _check_size(grads[i], (p.nz, p.nx), f"grad[{i}]")
        _check_size(misfits[i], (), f"misfit[{i}]")
    V = ctypes.c_void_p * n
    arr = (Problem * n)(*problems)

    def ptrs(ts):
        return V(*[_ptr(t) for t in ts])
    keep = [ptrs(models), ptrs(wavelets), ptrs(srcs), ptrs(recs), ptrs(d_obs), ptrs(grads),
            ptrs(misfits), V(*[ctypes.c_void_p(w.data_ptr()) for w in ws]),
            (ctypes.c_size_t * n)(*[w.numel() for w in ws])]
    args = [ctypes.cast(arr, ctypes.c_void_p)] + [ctypes.cast(k, ctypes.c_void_p) for k in keep]
    rc = _lib.sweep_gradient_batch(n, *args, _stream(stream))
    if rc != OK:
        raise SweepError(rc, "sweep_gradient_batch")
    if sync and not getattr(_capture_state, "on", False):
        for w in ws:
            st = status(w, stream)
            if st != OK:
                raise SweepError(st, "sweep_gradient_batch")
    return grads, misfits


def sweep_forward_batch(problems, models, wavelets, srcs, recs, data=None, ws=None,
                        stream=None, sync=True):
    """Acoustic forward runs of several problems in one call
    (sweep_forward_batch); returns the list of data tensors."""
    n = len(problems)
    if not (len(models) == len(wavelets) == len(srcs) == len(recs) == n):
        raise ValueError("sweep_forward_batch: one entry per problem in every list")
    if n == 0:
        return []
    dev = models[0].device
    data = list(data) if data is not None else [
        torch.empty((p.nshot, 1, p.nrec, p.nt), dtype=torch.float32, device=dev)
        for p in problems]
    ws = list(ws) if ws is not None else [
        alloc_workspace(p, MODE_FORWARD, dev) for p in problems]
    for i, p in enumerate(problems):
        if p.physics != ACOUSTIC:
            raise SweepError(EUNSUPPORTED, "sweep_forward_batch")
        for t, dt, name in ((models[i], torch.float32, "model"),
                            (wavelets[i], torch.float32, "wavelet"),
                            (srcs[i], torch.int32, "src"), (recs[i], torch.int32, "rec"),
                            (data[i], torch.float32, "data")):
            _check_dtype(t, dt, f"{name}[{i}]")
        _check_inputs(p, models[i], wavelets[i], srcs[i], recs[i])
        _check_size(data[i], (p.nshot, 1, p.nrec, p.nt), f"data[{i}]")
    V = ctypes.c_void_p * n
    arr = (Problem * n)(*problems)

    def ptrs(ts):
        return V(*[_ptr(t) for t in ts])
    keep = [ptrs(models), ptrs(wavelets), ptrs(srcs), ptrs(recs), ptrs(data),
            V(*[ctypes.c_void_p(w.data_ptr()) for w in ws]),
            (ctypes.c_size_t * n)(*[w.numel() for w in ws])]
    args = [ctypes.cast(arr, ctypes.c_void_p)] + [ctypes.cast(k, ctypes.c_void_p) for k in keep]
    rc = _lib.sweep_forward_batch(n, *args, _stream(stream))
    if rc != OK:
        raise SweepError(rc, "sweep_forward_batch")
    if sync and not getattr(_capture_state, "on", False):
        for w in ws:
            st = status(w, stream)
            if st != OK:
                raise SweepError(st, "sweep_forward_batch")
    return data


_capture_state = threading.local()


class Graph:
    """A recorded sequence of library calls (``capture``), replayed with
    ``launch``.  The recorded calls' tensors are reused at every replay:
    keep them alive and write new inputs into them in place."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @property
    def kernels(self) -> int:
        return int(_lib.sweep_graph_kernels(self._h))

    def launch(self, stream=None) -> None:
        if not self._h:
            raise ValueError("sweep.Graph: closed")
        rc = _lib.sweep_graph_launch(self._h, _stream(stream))
        if rc != OK:
            raise SweepError(rc, "sweep_graph_launch")

    def close(self) -> None:
        """Frees the graph; no replay of it may be pending."""
        if self._h:
            _lib.sweep_graph_destroy(self._h)
            self._h = ctypes.c_void_p(None)


class _Capture:
    graph: Graph | None = None


@contextlib.contextmanager
def capture(stream: torch.cuda.Stream):
    """Records the library calls made on ``stream`` by this thread inside the
    block into a ``Graph`` (``with capture(s) as c: ...; c.graph.launch(s)``).
    Inside the block, pass every output and workspace tensor explicitly (no
    allocation may happen during a capture) and ``stream=stream``; the
    status check of the calls is skipped (read it after a replay with
    ``status``).  ``stream`` must not be the legacy default stream."""
    if stream is None or stream.cuda_stream == 0:
        raise ValueError("sweep.capture: needs a non-default torch.cuda.Stream")
    stream.wait_stream(torch.cuda.current_stream(stream.device))
    rc = _lib.sweep_capture_begin(ctypes.c_void_p(stream.cuda_stream))
    if rc != OK:
        raise SweepError(rc, "sweep_capture_begin")
    cap = _Capture()
    _capture_state.on = True
    ok = False
    try:
        yield cap
        ok = True
    finally:
        _capture_state.on = False
        h = ctypes.c_void_p(None)
        rc = _lib.sweep_capture_end(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if ok:
            if rc != OK:
                raise SweepError(rc, "sweep_capture_end")
            cap.graph = Graph(h.value)
        elif h.value:
            _lib.sweep_graph_destroy(h)


_dot_ws = {}


def sweep_dot(a, b, out=None, stream=None):
    """FP64 sum(a * b) of two float32 CUDA tensors, as a device float64 scalar.

    The partial sums go to one scratch buffer per device, allocated on the
    first call and shared by later calls: calls on different streams must
    not overlap on the GPU (pass sweep_dot's C workspace yourself for that)."""
    _check_dtype(a, torch.float32, "a")
    _check_dtype(b, torch.float32, "b")
    if a.numel() != b.numel():
        raise ValueError("sweep_dot: size mismatch")
    dev = a.device
    if b.device != dev:
        raise ValueError("sweep_dot: a and b on different devices")
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=dev)
    _check_dtype(out, torch.float64, "out")
    if out.numel() != 1:
        raise ValueError("sweep_dot: out must be a one-element float64 tensor")
    key = (dev.index if dev.index is not None else torch.cuda.current_device())
    ws = _dot_ws.get(key)
    if ws is None:
        ws = torch.empty(int(_lib.sweep_dot_workspace_bytes()), dtype=torch.uint8, device=dev)
        _dot_ws[key] = ws
    w, wn = _ws_args(ws)
    rc = _lib.sweep_dot(_ptr(a), _ptr(b), ctypes.c_int64(a.numel()), _ptr(out), w, wn,
                        _stream(stream))
    if rc != OK:
        raise SweepError(rc, "sweep_dot")
    return out
