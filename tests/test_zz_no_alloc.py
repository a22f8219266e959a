"""sweep_dot_noalloc: the FP64 dot product for callers that cannot allocate
device memory (for example a plugin whose host application owns the whole
device-memory budget, or a loop that must not allocate after start-up).

It keeps its partial sums in a fixed device array inside the library instead
of a caller-provided workspace.  Called here directly through the C ABI and
compared with sweep_dot (which uses a workspace) on two calls in a row, so
that a second call must not see anything the first one left behind.  The
file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_14189_gb300 import sweep
    return sweep


def _call(sw, a, b, n, out):
    st = torch.cuda.current_stream()
    return sw.lib().sweep_dot_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                      ctypes.c_int64(n), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(st.cuda_stream))


def test_noalloc_dot_matches_workspace_dot_twice(sw):
    torch.manual_seed(0)
    # second call is shorter: its result must not include the first call's
    # partial sums still sitting in the shared array
    for n in (3_000_017, 70_001):
        a = torch.randn(n, device="cuda", dtype=torch.float32)
        b = torch.randn(n, device="cuda", dtype=torch.float32)
        out = torch.full((), float("nan"), device="cuda", dtype=torch.float64)
        assert _call(sw, a, b, n, out) == sw.OK
        ref = sw.sweep_dot(a, b).item()
        got = out.item()
        host = float(np.dot(a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)))
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        assert abs(got - host) <= 1e-12 * abs(host), (got, host)


def test_noalloc_dot_edges(sw):
    a = torch.ones(10, device="cuda")
    out = torch.full((), 5.0, device="cuda", dtype=torch.float64)
    assert _call(sw, a, a, 0, out) == sw.OK  # empty: sum is 0
    assert out.item() == 0.0
    # above the fixed capacity: rejected before any launch
    assert _call(sw, a, a, sw.DOT_NOALLOC_MAX_N + 1, out) == sw.ETOOBIG
    assert sw.strerror(sw.ETOOBIG).startswith("size above")
