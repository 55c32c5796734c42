"""Parity measures of the GPU tests against the FP64 oracle.

Each comparison is held to its stated tolerance twice: as a whole-array
relative L2 error, and element by element as max |gpu - oracle| / max |oracle|,
so that a wrong value in a few pixels, rays or voxels cannot hide under the
norm of the rest."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def assert_close(got, want, tol, elem_tol=None, what=""):
    """rel-L2 <= tol and max |got - want| / max |want| <= elem_tol (default tol)."""
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    r, m = rel_l2(got, want), max_rel(got, want)
    et = tol if elem_tol is None else elem_tol
    assert r <= tol and m <= et, "%s: rel-L2 %.3e (bound %.1e), per-element %.3e (bound %.1e)" % (
        what, r, tol, m, et)
    return r, m
