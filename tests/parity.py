"""Comparison helpers for CUDA-vs-oracle parity (test code only).

Relative-error convention: rho and T pointwise |d|/|ref|; U and q
field-normalised max|d| / max|ref field| (they pass through zero).
Per-component errors normalise each of Ux, Uy, Uz, qx, qy, qz by its own
largest magnitude instead (floored at a fraction of the field's, so that a
component that is zero by symmetry is compared on the field's scale).
Solid cells are excluded.
"""
import numpy as np


def field_errors(got, ref, solid=None):
    got = np.asarray(got).reshape(8, -1)
    ref = np.asarray(ref).reshape(8, -1)
    mask = np.ones(got.shape[1], bool) if solid is None else ~np.asarray(solid, bool).reshape(-1)
    g, r = got[:, mask], ref[:, mask]
    err = {}
    err["rho"] = float(np.max(np.abs(g[0] - r[0]) / np.abs(r[0])))
    err["T"] = float(np.max(np.abs(g[4] - r[4]) / np.abs(r[4])))
    for name, sl in (("U", slice(1, 4)), ("q", slice(5, 8))):
        scale = max(np.max(np.abs(r[sl])), 1e-300)
        err[name] = float(np.max(np.abs(g[sl] - r[sl])) / scale)
    return err


def assert_fields_close(got, ref, tol, solid=None, what=""):
    err = field_errors(got, ref, solid)
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, "%s: relative errors above %g: %s (all: %s)" % (what, tol, bad, err)
    return err


def assert_rho_w_close(got, ref, tol):
    got = np.asarray(got).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    wall = ref != 0.0
    assert np.array_equal(wall, got != 0.0), "wall-face sets differ"
    if wall.any():
        rel = np.max(np.abs(got[wall] - ref[wall]) / np.abs(ref[wall]))
        assert rel <= tol, "rho_w relative error %g > %g" % (rel, tol)


def component_errors(got, ref, solid=None, floor=1e-2):
    """max|d| / max(max|ref component|, floor * max|ref field|) for each
    component of U and q."""
    got = np.asarray(got).reshape(8, -1)
    ref = np.asarray(ref).reshape(8, -1)
    mask = np.ones(got.shape[1], bool) if solid is None else ~np.asarray(solid, bool).reshape(-1)
    g, r = got[:, mask], ref[:, mask]
    out = {}
    for name, rows in (("U", (1, 2, 3)), ("q", (5, 6, 7))):
        field = max(np.max(np.abs(r[rows[0]:rows[-1] + 1])), 1e-300)
        for axis, q in zip("xyz", rows):
            scale = max(np.max(np.abs(r[q])), floor * field)
            out[name + axis] = float(np.max(np.abs(g[q] - r[q])) / scale)
    return out


def assert_components_close(got, ref, tol, solid=None, what=""):
    err = component_errors(got, ref, solid)
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, "%s: per-component errors above %g: %s (all: %s)" % (what, tol, bad, err)
    return err
