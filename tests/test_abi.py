"""The C-ABI library builds, loads and exports every symbol include/sweep.h
declares; host-side validation rejects bad arguments before any launch.
No GPU is needed: nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

from paper_2604_14189_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(header="sweep.h"):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(sweep_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def _headers():
    return sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    assert _headers() == ["sweep.h", "unet.h"]
    for h in _headers():
        names = _declared_functions(h)
        assert len(names) >= 8, h
        for n in names:
            assert hasattr(lib, n), (h, n)


def test_binding_lists_every_symbol():
    from paper_2604_14189_gb300 import sweep, unet
    assert set(sweep.EXPORTS) == set(_declared_functions("sweep.h"))
    assert set(unet.EXPORTS) == set(_declared_functions("unet.h"))


def test_unet_host_validation():
    """U-Net entry points: parameter count, workspace sizes and host-side
    rejection of bad shapes, before any launch."""
    from paper_2604_14189_gb300 import sweep, unet
    from oracle import unet as ounet
    L = sweep.lib()
    assert L.sweep_unet_param_count() == unet.PARAMS == ounet.param_count()
    ok = unet.shape(2, 256, 256, 2)
    inf = unet.workspace_bytes(ok, False)
    trn = unet.workspace_bytes(ok, True)
    assert 0 < inf < trn
    for bad in ((0, 256, 256, 2), (1, 100, 256, 2), (1, 256, 192, 2), (1, 256, 64, 2),
                (1, 256, 256, 0), (1, 256, 256, 33), (1, 64, 128, 1)):
        assert unet.workspace_bytes(unet.shape(*bad), True) == 0, bad
    fake = ctypes.c_void_p(256)
    assert L.sweep_unet_forward(ctypes.byref(unet.shape(0, 256, 256, 2)), fake, fake, fake,
                                fake, 1 << 40, None) == sweep.EINVAL
    assert L.sweep_unet_forward(ctypes.byref(ok), fake, fake, fake, None, 1 << 40,
                                None) == sweep.EWORKSPACE
    assert L.sweep_unet_forward(ctypes.byref(ok), fake, fake, fake, fake, inf - 1,
                                None) == sweep.EWORKSPACE
    assert L.sweep_unet_gradient(ctypes.byref(ok), fake, fake, None, fake, fake, fake, fake,
                                 1 << 40, None) == sweep.EINVAL
    # single-layer kernels: channel counts and tile shapes
    assert L.sweep_unet_conv3x3(1, 128, 128, 48, 32, fake, fake, None, 1, None, fake, fake,
                                256, None) == sweep.EINVAL
    assert L.sweep_unet_conv3x3(1, 128, 128, 32, 512, fake, fake, None, 1, None, fake, fake,
                                256, None) == sweep.EINVAL
    assert L.sweep_unet_conv3x3(1, 12, 16, 32, 32, fake, fake, None, 1, None, fake, fake,
                                256, None) == sweep.EINVAL
    assert L.sweep_unet_conv3x3(1, 128, 128, 32, 32, fake, fake, None, 2, None, fake, fake,
                                256, None) == sweep.EINVAL  # mask op without a mask
    assert L.sweep_unet_wgrad_workspace_bytes(1, 128, 128, 32, 32) > 0
    assert L.sweep_unet_wgrad_workspace_bytes(1, 128, 100, 32, 32) == 0
    assert L.sweep_unet_adam(fake, fake, fake, fake, 10, 0, 1e-3, 0.9, 0.999, 1e-8,
                             None) == sweep.EINVAL


def _prob(sweep, **kw):
    base = dict(nz=20, nx=30, pml=5, dx=10.0, dt=1e-3, nt=10, nshot=2, nrec=3)
    base.update(kw)
    return sweep.problem(**base)


def test_workspace_size_and_validation():
    from paper_2604_14189_gb300 import sweep
    p = _prob(sweep)
    fwd = sweep.workspace_bytes(p, sweep.MODE_FORWARD)
    adj = sweep.workspace_bytes(p, sweep.MODE_ADJOINT)
    grd = sweep.workspace_bytes(p, sweep.MODE_GRADIENT)
    assert 0 < fwd < grd and 0 < adj < grd
    for bad in (dict(nz=0), dict(nx=-1), dict(pml=-1), dict(nt=0), dict(nshot=-1),
                dict(dx=0.0), dict(dt=-1.0), dict(dx=float("nan")),
                # one shot's field beyond 32-bit indices on the padded row pitch
                dict(nz=46341, nx=46341, pml=0, nshot=1),
                # (tile, shot) units beyond 32 bits
                dict(nz=20000, nx=20000, pml=0, nshot=65535),
                dict(nshot=65536),
                # a flag bit the library does not define
                dict(flags=0x20), dict(flags=-1)):
        q = _prob(sweep, **bad)
        assert sweep.lib().sweep_workspace_bytes(ctypes.byref(q), 0) == 0, bad
    assert sweep.lib().sweep_workspace_bytes(ctypes.byref(p), 7) == 0
    # the tuning flag changes neither validity nor the workspace
    q = _prob(sweep, flags=sweep.F_ROWS16)
    assert sweep.lib().sweep_workspace_bytes(ctypes.byref(q), 2) == grd
    # the largest sizes still accepted
    big = _prob(sweep, nz=46000, nx=46000, pml=0, nshot=1)
    assert sweep.lib().sweep_workspace_bytes(ctypes.byref(big), 0) > 0


def test_host_errors_before_launch():
    """Invalid problems, NULL or small workspaces are rejected on the host."""
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    p = _prob(sweep)
    fake = ctypes.c_void_p(256)  # never dereferenced: rejected first
    q = _prob(sweep, nz=0)
    assert L.sweep_forward(ctypes.byref(q), fake, fake, fake, fake, fake, fake,
                           1 << 30, None) == sweep.EINVAL
    assert L.sweep_forward(ctypes.byref(p), fake, fake, fake, fake, fake, None, 1 << 30,
                           None) == sweep.EWORKSPACE
    assert L.sweep_forward(ctypes.byref(p), fake, fake, fake, fake, fake, fake, 16,
                           None) == sweep.EWORKSPACE
    assert L.sweep_forward(ctypes.byref(p), fake, fake, fake, fake, fake,
                           ctypes.c_void_p(257), 1 << 30, None) == sweep.EWORKSPACE
    assert L.sweep_dot(None, None, -1, None, None, 0, None) == sweep.EINVAL
    assert sweep.strerror(sweep.ECFL).startswith("time step")


def test_null_arrays_rejected_before_device_work():
    """With a workspace that passes every host check, a NULL array is still
    reported as SWEEP_EINVAL before the call touches the device (on a host
    without a GPU, any device call would return SWEEP_ECUDA instead)."""
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    p = _prob(sweep)
    fake = ctypes.c_void_p(1 << 20)  # 256-byte aligned, never dereferenced
    big = 1 << 40
    V = None
    assert L.sweep_forward(ctypes.byref(p), V, fake, fake, fake, fake, fake, big,
                           None) == sweep.EINVAL
    assert L.sweep_forward(ctypes.byref(p), fake, V, fake, fake, fake, fake, big,
                           None) == sweep.EINVAL
    assert L.sweep_forward(ctypes.byref(p), fake, fake, fake, fake, V, fake, big,
                           None) == sweep.EINVAL
    assert L.sweep_adjoint(ctypes.byref(p), fake, fake, fake, fake, V, fake, big,
                           None) == sweep.EINVAL
    assert L.sweep_adjoint(ctypes.byref(p), fake, V, fake, fake, fake, fake, big,
                           None) == sweep.EINVAL
    assert L.sweep_gradient(ctypes.byref(p), fake, fake, fake, fake, fake, V, fake, fake,
                            fake, big, None) == sweep.EINVAL
    assert L.sweep_gradient(ctypes.byref(p), fake, fake, fake, fake, V, fake, fake, fake,
                            fake, big, None) == sweep.EINVAL
    el = _prob(sweep, physics=sweep.ELASTIC)
    assert L.sweep_gradient(ctypes.byref(el), fake, fake, fake, fake, fake, fake, fake,
                            fake, fake, big, None) == sweep.EUNSUPPORTED  # illum, elastic


def test_capture_rejects_bad_arguments(lib):
    """Host-side checks of the graph calls, before any CUDA call: the legacy
    default stream cannot be captured, and ending or launching needs a
    capture or a graph."""
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    assert L.sweep_capture_begin(None) == sweep.EINVAL
    h = ctypes.c_void_p(None)
    assert L.sweep_capture_end(None, ctypes.byref(h)) == sweep.EINVAL
    assert L.sweep_capture_end(ctypes.c_void_p(1), None) == sweep.EINVAL
    assert L.sweep_graph_launch(None, None) == sweep.EINVAL
    assert L.sweep_graph_kernels(None) == sweep.EINVAL
    L.sweep_graph_destroy(None)  # no-op


def test_wait_timeout_diagnostic_checks_workspace(lib):
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    assert L.sweep_check_wait_timeout(None, 1024, None) == sweep.EWORKSPACE
    assert L.sweep_check_wait_timeout(ctypes.c_void_p(256), 2, None) == sweep.EWORKSPACE
    assert L.sweep_check_wait_timeout(ctypes.c_void_p(257), 1024, None) == sweep.EWORKSPACE
    assert L.sweep_check_barrier_timeout(None, 1024, None) == sweep.EWORKSPACE
    assert L.sweep_check_barrier_timeout(ctypes.c_void_p(256), 64, None) == sweep.EWORKSPACE
    assert L.sweep_check_barrier_timeout(ctypes.c_void_p(257), 1024, None) == sweep.EWORKSPACE


def test_one_launch_flag_rules():
    """SWEEP_F_ONE_LAUNCH: accepted by validation (same workspace size);
    with an illumination request or in sweep_adjoint the call is refused
    before anything is launched; a batch whose problems disagree on the flag
    is refused too."""
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    p = _prob(sweep)
    q = _prob(sweep, flags=sweep.F_ONE_LAUNCH)
    for mode in (0, 1, 2):
        assert (L.sweep_workspace_bytes(ctypes.byref(q), mode)
                == L.sweep_workspace_bytes(ctypes.byref(p), mode))
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: refused before a launch
    big = ctypes.c_size_t(1 << 40)
    assert L.sweep_gradient(ctypes.byref(q), fake, fake, fake, fake, fake, fake, fake, fake,
                            fake, big, None) == sweep.EUNSUPPORTED
    assert L.sweep_adjoint(ctypes.byref(q), fake, fake, fake, fake, fake, fake, big,
                           None) == sweep.EUNSUPPORTED
    probs = (sweep.Problem * 2)(p, q)
    ptrs = (ctypes.c_void_p * 2)(fake, fake)
    sizes = (ctypes.c_size_t * 2)(1 << 40, 1 << 40)
    assert L.sweep_forward_batch(2, probs, ptrs, ptrs, ptrs, ptrs, ptrs, ptrs, sizes,
                                 None) == sweep.EINVAL


def test_deterministic_flag_rules():
    """SWEEP_F_DETERMINISTIC: same workspace; refused with the time-loop
    kernels; a batch whose problems disagree on it is refused."""
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    p = _prob(sweep)
    d = _prob(sweep, flags=sweep.F_DETERMINISTIC)
    for mode in (0, 1, 2):
        assert (L.sweep_workspace_bytes(ctypes.byref(d), mode)
                == L.sweep_workspace_bytes(ctypes.byref(p), mode))
    both = _prob(sweep, flags=sweep.F_DETERMINISTIC | sweep.F_ONE_LAUNCH)
    fake = ctypes.c_void_p(1 << 20)
    big = ctypes.c_size_t(1 << 40)
    assert L.sweep_forward(ctypes.byref(both), fake, fake, fake, fake, fake, fake, big,
                           None) == sweep.EUNSUPPORTED
    assert L.sweep_gradient(ctypes.byref(both), fake, fake, fake, fake, fake, fake, fake, None,
                            fake, big, None) == sweep.EUNSUPPORTED
    probs = (sweep.Problem * 2)(p, d)
    ptrs = (ctypes.c_void_p * 2)(fake, fake)
    sizes = (ctypes.c_size_t * 2)(1 << 40, 1 << 40)
    assert L.sweep_gradient_batch(2, probs, ptrs, ptrs, ptrs, ptrs, ptrs, ptrs, ptrs, ptrs,
                                  sizes, None) == sweep.EINVAL


def test_binding_rejects_wrong_sizes_before_any_call():
    """The binding checks every tensor's element count against the problem
    before it reaches the C ABI (which sees only pointers); CPU tensors are
    enough: the size check comes before the device check."""
    import torch
    from paper_2604_14189_gb300 import sweep
    p = _prob(sweep)  # nz 20, nx 30, nt 10, 2 shots, 3 receivers
    f32, i32 = torch.float32, torch.int32
    good = dict(model=torch.zeros(20, 30, dtype=f32), wavelet=torch.zeros(2, 10, dtype=f32),
                src=torch.zeros(2, 2, dtype=i32), rec=torch.zeros(2, 3, 2, dtype=i32))
    bad = dict(model=torch.zeros(20, 29, dtype=f32), wavelet=torch.zeros(2, 9, dtype=f32),
               src=torch.zeros(1, 2, dtype=i32), rec=torch.zeros(2, 2, 2, dtype=i32))
    for k in bad:
        args = dict(good, **{k: bad[k]})
        with pytest.raises(ValueError, match=k):
            sweep.sweep_forward(p, args["model"], args["wavelet"], args["src"], args["rec"])
    with pytest.raises(ValueError, match="data"):
        sweep.sweep_forward(p, **good, data=torch.zeros(2, 1, 3, 9, dtype=f32))
    with pytest.raises(ValueError, match="d_obs"):
        sweep.sweep_gradient(p, good["model"], good["wavelet"], good["src"], good["rec"],
                             torch.zeros(2, 1, 3, 11, dtype=f32))
    with pytest.raises(ValueError, match="grad"):
        sweep.sweep_gradient(p, good["model"], good["wavelet"], good["src"], good["rec"],
                             torch.zeros(2, 1, 3, 10, dtype=f32),
                             grad=torch.zeros(20, 31, dtype=f32))
    with pytest.raises(ValueError, match="adj_data"):
        sweep.sweep_adjoint(p, good["model"], torch.zeros(2, 3, 11, dtype=f32), good["src"],
                            good["rec"])
    # a padded model has the padded size
    q = _prob(sweep, flags=sweep.F_PADDED_MODEL)
    with pytest.raises(ValueError, match="model"):
        sweep.sweep_forward(q, good["model"], good["wavelet"], good["src"], good["rec"])


def test_gradient_batch_host_checks(lib):
    """sweep_gradient_batch checks every problem on the host before any
    launch: bad counts, elastic problems, a workspace shared by two problems,
    and missing pointers."""
    from paper_2604_14189_gb300 import sweep
    L = sweep.lib()
    V = ctypes.c_void_p
    assert L.sweep_gradient_batch(-1, *([None] * 11)) == sweep.EINVAL
    assert L.sweep_gradient_batch(0, *([None] * 11)) == sweep.OK
    assert L.sweep_gradient_batch(2, *([None] * 11)) == sweep.EINVAL
    p = _prob(sweep)
    q = _prob(sweep)
    need = sweep.workspace_bytes(p, sweep.MODE_GRADIENT)
    fake = V(1 << 20)  # never dereferenced: every check fails before a launch

    def call(probs, wss, sizes, model=fake):
        n = len(probs)
        arr = (sweep.Problem * n)(*probs)
        ptrs = (V * n)(*([model] * n))
        wsa = (V * n)(*wss)
        sza = (ctypes.c_size_t * n)(*sizes)
        args = [ctypes.cast(arr, V)] + [ctypes.cast(ptrs, V)] * 7 + [ctypes.cast(wsa, V),
                                                                   ctypes.cast(sza, V)]
        return L.sweep_gradient_batch(n, *args, None)

    el = _prob(sweep, physics=sweep.ELASTIC)
    assert call([p, el], [V(256 * 4096), V(512 * 4096)], [need, need]) == sweep.EUNSUPPORTED
    assert call([p, q], [V(256 * 4096), V(256 * 4096)], [need, need]) == sweep.EWORKSPACE
    assert call([p, q], [V(256 * 4096), V(512 * 4096)], [need, need - 1]) == sweep.EWORKSPACE
    assert call([p, q], [V(256 * 4096), V(512 * 4096)], [need, need], model=V(0)) == sweep.EINVAL


def test_dot_binding_checks_out_before_any_launch():
    """sweep_dot writes 8 bytes to `out`: a float32 or multi-element `out`
    is rejected on the host, as are mismatched sizes."""
    import torch

    from paper_2604_14189_gb300 import sweep
    a = torch.zeros(4, dtype=torch.float32)
    with pytest.raises(TypeError, match="out"):
        sweep.sweep_dot(a, a, out=torch.zeros((), dtype=torch.float32))
    with pytest.raises(ValueError, match="out"):
        sweep.sweep_dot(a, a, out=torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="size"):
        sweep.sweep_dot(a, torch.zeros(5, dtype=torch.float32))


def test_profile_classes_match_the_header(lib):
    """The binding's kernel-class constants are the header's SWEEP_K_*
    values, and a class past SWEEP_K_COUNT is rejected on the host."""
    from paper_2604_14189_gb300 import sweep
    txt = open(os.path.join(ROOT, "include", "sweep.h")).read()
    vals = {k: int(v) for k, v in re.findall(r"\bSWEEP_K_(\w+)\s*=\s*(\d+)", txt)}
    for name in ("AC_FWD", "AC_BWD", "EL_VEL", "EL_STR", "AC_FWD_LOOP", "AC_BWD_LOOP",
                 "EL_ADJ"):
        assert getattr(sweep, "K_" + name) == vals[name], name
    assert sorted(v for k, v in vals.items() if k != "COUNT") == list(range(vals["COUNT"]))
    ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
    lib.sweep_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]
    assert lib.sweep_profile_read(vals["COUNT"], ctypes.byref(ms), ctypes.byref(n)) \
        == sweep.EINVAL
    assert lib.sweep_profile_read(-1, ctypes.byref(ms), ctypes.byref(n)) == sweep.EINVAL
