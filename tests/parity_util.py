"""Comparison helpers of the GPU parity tests (no solver arithmetic).

Beside the global relative L2 of a record or a gradient, the parity tests
check every trace on its own and the gradient in regions where an error
could hide under the global norm: the band inside the interior edge (where
the backward pass restores the forward wavefield's ring) and the
neighbourhood of every source (where the imaging condition adds the source
term and the gradient is largest)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def worst_trace(d, ref, floor=1e-3):
    """Largest per-trace relative L2 over [..., nt] records.  A trace whose
    reference norm is below `floor` of the largest trace norm (silent: the
    wave has not reached it) is measured against that floor instead."""
    d = np.asarray(d, dtype=np.float64).reshape(-1, np.shape(d)[-1])
    ref = np.asarray(ref, dtype=np.float64).reshape(-1, np.shape(ref)[-1])
    nr = np.linalg.norm(ref, axis=1)
    den = np.maximum(nr, floor * nr.max())
    return float(np.max(np.linalg.norm(d - ref, axis=1) / den))


def region_errors(g, gref, src, band=4, half=4, floor=1e-3):
    """Relative L2 of g in the `band`-cell band inside the interior edge and
    in the (2 half + 1)^2 neighbourhood of each distinct source cell
    (interior coordinates (z, x)).  A region whose reference norm is below
    `floor` of the whole gradient's norm (a shot whose receivers the wave
    has not reached leaves its source region at rounding level) is measured
    against that floor instead."""
    g = np.asarray(g, dtype=np.float64)
    gref = np.asarray(gref, dtype=np.float64)
    nz, nx = gref.shape
    scale = floor * np.linalg.norm(gref)

    def err(a, b):
        return np.linalg.norm(a - b) / max(np.linalg.norm(b), scale, 1e-300)

    m = np.zeros((nz, nx), dtype=bool)
    m[:band] = m[-band:] = True
    m[:, :band] = m[:, -band:] = True
    out = {"band": err(g[m], gref[m])}
    for sz, sx in np.unique(np.asarray(src).reshape(-1, 2), axis=0):
        z0, z1 = max(sz - half, 0), min(sz + half + 1, nz)
        x0, x1 = max(sx - half, 0), min(sx + half + 1, nx)
        out[f"src({sz},{sx})"] = err(g[z0:z1, x0:x1], gref[z0:z1, x0:x1])
    return out


def assert_gradient(g, gref, src, tol=1e-3):
    """Global relative L2 and every region of region_errors within tol."""
    err = rel(g, gref)
    assert err <= tol, err
    bad = {k: e for k, e in region_errors(g, gref, src).items() if not e <= tol}
    assert not bad, bad
