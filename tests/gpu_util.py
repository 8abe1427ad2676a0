"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def max_rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# Element-wise companion of a relative-L2 bound.  An error spread over the
# field (rounding) has max|d| below about 6 rms(d) on up to 2^26 points (the
# tail of a Gaussian), and max|ref| >= rms(ref), so a result within `tol` in
# relative L2 meets max|d| <= 6 tol max|ref|.  An error confined to a few
# points (a Nyquist row or column, a tile edge, one field of a batch) can stay
# under the L2 bound while failing this one.
ELEM_FACTOR = 6.0


def check(got, ref, tol, elem=None):
    """Assert rel L2 <= tol and max|got - ref| <= elem * max|ref| (elem
    defaults to ELEM_FACTOR * tol); returns both measured figures."""
    e2, em = rel_l2(got, ref), max_rel(got, ref)
    elem = ELEM_FACTOR * tol if elem is None else elem
    assert e2 <= tol and em <= elem, \
        f"rel L2 {e2:.3g} (bound {tol:.3g}), max |d| / max |ref| {em:.3g} (bound {elem:.3g})"
    return e2, em


EPS = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}
