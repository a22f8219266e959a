"""Thin ctypes binding of the U-Net preconditioner's C ABI (``include/unet.h``,
in ``libsweep.so``).

Argument marshalling only: the forward pass, the backward pass and Adam run
in the library's CUDA kernels (the convolutions on the tcgen05 tensor
cores).  Tensors must be contiguous CUDA tensors; BF16 arrays are
``torch.bfloat16``.  No CPU fallback: importing fails without the library.
"""
from __future__ import annotations

import ctypes

import torch

from . import sweep

PARAMS = 2148993
EXPORTS = ("sweep_unet_param_count", "sweep_unet_workspace_bytes", "sweep_unet_forward",
           "sweep_unet_gradient", "sweep_unet_adam", "sweep_unet_conv3x3",
           "sweep_unet_wgrad_workspace_bytes", "sweep_unet_conv3x3_wgrad")
OP_NONE, OP_RELU, OP_MASK = 0, 1, 2


class Shape(ctypes.Structure):
    """Mirror of ``sweep_unet_shape``."""
    _fields_ = [("batch", ctypes.c_int32), ("height", ctypes.c_int32),
                ("width", ctypes.c_int32), ("in_ch", ctypes.c_int32)]


def _setup(lib):
    vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32
    S = ctypes.POINTER(Shape)
    lib.sweep_unet_param_count.argtypes = []
    lib.sweep_unet_param_count.restype = ctypes.c_longlong
    lib.sweep_unet_workspace_bytes.argtypes = [S, ctypes.c_int]
    lib.sweep_unet_workspace_bytes.restype = sz
    lib.sweep_unet_forward.argtypes = [S, vp, vp, vp, vp, sz, vp]
    lib.sweep_unet_forward.restype = ctypes.c_int
    lib.sweep_unet_gradient.argtypes = [S, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sweep_unet_gradient.restype = ctypes.c_int
    lib.sweep_unet_adam.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, i32, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]
    lib.sweep_unet_adam.restype = ctypes.c_int
    lib.sweep_unet_conv3x3.argtypes = [i32] * 5 + [vp, vp, vp, i32, vp, vp, vp, sz, vp]
    lib.sweep_unet_conv3x3.restype = ctypes.c_int
    lib.sweep_unet_wgrad_workspace_bytes.argtypes = [i32] * 5
    lib.sweep_unet_wgrad_workspace_bytes.restype = sz
    lib.sweep_unet_conv3x3_wgrad.argtypes = [i32] * 5 + [vp, vp, vp, vp, sz, vp]
    lib.sweep_unet_conv3x3_wgrad.restype = ctypes.c_int
    return lib


_lib = _setup(sweep.lib())


def _ptr(t):
    return sweep._ptr(t)


def _check(t, dt, shape, name):
    if t.dtype != dt:
        raise TypeError(f"unet: {name} must be {dt}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"unet: {name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def shape(batch, height, width, in_ch) -> Shape:
    return Shape(batch, height, width, in_ch)


def workspace_bytes(s: Shape, training: bool) -> int:
    return int(_lib.sweep_unet_workspace_bytes(ctypes.byref(s), 1 if training else 0))


def alloc_workspace(s: Shape, training: bool, device=None) -> torch.Tensor:
    n = workspace_bytes(s, training)
    if n == 0:
        raise sweep.SweepError(sweep.EINVAL, "sweep_unet_workspace_bytes")
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def _run(rc, ws, where, stream):
    if rc != sweep.OK:
        raise sweep.SweepError(rc, where)
    st = sweep.status(ws, stream) if ws is not None else sweep.OK
    if st != sweep.OK:
        raise sweep.SweepError(st, where)


def forward(s: Shape, theta, inp, out=None, ws=None, stream=None, sync=True):
    """Network output [B][H][W] (float32) for inp [B][H][W][in_ch]."""
    _check(theta, torch.float32, (PARAMS,), "theta")
    _check(inp, torch.float32, (s.batch, s.height, s.width, s.in_ch), "input")
    if out is None:
        out = torch.empty((s.batch, s.height, s.width), dtype=torch.float32, device=inp.device)
    if ws is None:
        ws = alloc_workspace(s, False, inp.device)
    rc = _lib.sweep_unet_forward(ctypes.byref(s), _ptr(theta), _ptr(inp), _ptr(out),
                                 _ptr(ws), ws.numel(), sweep._stream(stream))
    _run(rc, ws if sync else None, "sweep_unet_forward", stream)
    return out


def gradient(s: Shape, theta, inp, target, grad=None, out=None, loss=None, ws=None,
             stream=None, sync=True):
    """(loss [float64 scalar], grad [PARAMS], output) of the MSE loss."""
    _check(theta, torch.float32, (PARAMS,), "theta")
    _check(inp, torch.float32, (s.batch, s.height, s.width, s.in_ch), "input")
    _check(target, torch.float32, (s.batch, s.height, s.width), "target")
    dev = inp.device
    grad = torch.empty(PARAMS, dtype=torch.float32, device=dev) if grad is None else grad
    out = torch.empty((s.batch, s.height, s.width), dtype=torch.float32,
                      device=dev) if out is None else out
    loss = torch.empty((), dtype=torch.float64, device=dev) if loss is None else loss
    if ws is None:
        ws = alloc_workspace(s, True, dev)
    rc = _lib.sweep_unet_gradient(ctypes.byref(s), _ptr(theta), _ptr(inp), _ptr(target),
                                  _ptr(out), _ptr(loss), _ptr(grad), _ptr(ws), ws.numel(),
                                  sweep._stream(stream))
    _run(rc, ws if sync else None, "sweep_unet_gradient", stream)
    return loss, grad, out


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """In-place Adam update of theta (and its moments m, v)."""
    for t, name in ((theta, "theta"), (grad, "grad"), (m, "m"), (v, "v")):
        _check(t, torch.float32, (theta.numel(),), name)
    rc = _lib.sweep_unet_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(),
                              int(step), float(lr), float(beta1), float(beta2), float(eps),
                              sweep._stream(stream))
    if rc != sweep.OK:
        raise sweep.SweepError(rc, "sweep_unet_adam")


def conv3x3(x, w, bias=None, op=OP_NONE, mask=None, out=None, stream=None):
    """One tensor-core 3 x 3 convolution: x [B][H][W][cin] bf16,
    w [cout][9][cin] bf16, bias [cout] float32 -> out [B][H][W][cout] bf16."""
    B, H, W, cin = x.shape
    cout = w.shape[0]
    _check(x, torch.bfloat16, (B, H, W, cin), "x")
    _check(w, torch.bfloat16, (cout, 9, cin), "w")
    if bias is not None:
        _check(bias, torch.float32, (cout,), "bias")
    if mask is not None:
        _check(mask, torch.bfloat16, (B, H, W, cout), "mask")
    if out is None:
        out = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device=x.device)
    ws = torch.zeros(256, dtype=torch.uint8, device=x.device)
    rc = _lib.sweep_unet_conv3x3(B, H, W, cin, cout, _ptr(x), _ptr(w), _ptr(bias), int(op),
                                 _ptr(mask), _ptr(out), _ptr(ws), ws.numel(),
                                 sweep._stream(stream))
    _run(rc, ws, "sweep_unet_conv3x3", stream)
    return out


def conv3x3_wgrad(x, dy, dw=None, stream=None):
    """Weight gradient [cout][9][cin] (float32) of conv3x3 for input x and
    output gradient dy (both bf16 NHWC)."""
    B, H, W, cin = x.shape
    cout = dy.shape[-1]
    _check(x, torch.bfloat16, (B, H, W, cin), "x")
    _check(dy, torch.bfloat16, (B, H, W, cout), "dy")
    if dw is None:
        dw = torch.empty((cout, 9, cin), dtype=torch.float32, device=x.device)
    n = int(_lib.sweep_unet_wgrad_workspace_bytes(B, H, W, cin, cout))
    if n == 0:
        raise sweep.SweepError(sweep.EINVAL, "sweep_unet_wgrad_workspace_bytes")
    ws = torch.empty(n, dtype=torch.uint8, device=x.device)
    rc = _lib.sweep_unet_conv3x3_wgrad(B, H, W, cin, cout, _ptr(x), _ptr(dy), _ptr(dw),
                                       _ptr(ws), ws.numel(), sweep._stream(stream))
    _run(rc, ws, "sweep_unet_conv3x3_wgrad", stream)
    return dw
