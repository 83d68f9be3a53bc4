"""Comparison helpers of the GPU parity tests (the oracle is the reference).

* ``rel``: relative L2 over all compared coefficients, ||a - b|| / ||b||;
* ``elem_max``: the largest per-element error ||a_e - b_e|| over the RMS
  per-element norm of b.  An error confined to a few elements (one color, the
  boundary edges, the ragged last tile of a color) is diluted by up to
  1/sqrt(elements) in the global norm; this measure sees it undiluted.
* ``check``: both at once.  The per-element bound is ELEM_FACTOR times the
  relative-L2 tolerance: for rounding-level differences spread over the mesh the
  ratio of the two measures is 4-6 (FP64 oracle against its extended build on
  the parity meshes).
"""

import numpy as np

ELEM_FACTOR = 10.0


def _f64(x):
    return np.asarray(x).astype(np.float64)


def rel(a, b) -> float:
    a, b = _f64(a), _f64(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def elem_max(a, b) -> float:
    a, b = _f64(a), _f64(b)
    n = a.shape[0]
    d = np.linalg.norm((a - b).reshape(n, -1), axis=1)
    s = np.linalg.norm(b.reshape(n, -1), axis=1)
    return float(d.max() / np.sqrt(np.mean(s * s)))


def check(a, b, tol, what: str = ""):
    """Assert rel(a, b) < tol and elem_max(a, b) < ELEM_FACTOR * tol; returns both."""
    e, m = rel(a, b), elem_max(a, b)
    assert e < tol, f"{what} relative L2 {e:.3e} >= {tol:.1e}"
    assert m < ELEM_FACTOR * tol, f"{what} per-element max {m:.3e} >= {ELEM_FACTOR * tol:.1e} (relative L2 {e:.3e})"
    return e, m


def fp64_vs_exact(got, ref64, refx, tol, what: str = ""):
    """FP64 parity against the oracle's extended-precision build.

    refx is the same right-hand side (or state change) evaluated with a wider
    significand: the exact result of the same inputs to far below FP64
    rounding.  ref64 is the FP64 oracle's value.  Where the terms of Eq. 2
    cancel to a much smaller sum (fine meshes, steep states), no FP64
    evaluation reaches tol against the exact result; the bound is then what the
    plain FP64 oracle itself reaches.  Both measures of ``check`` apply.
    Returns (GPU error, FP64 oracle error), relative L2 against refx."""
    e_gpu, e_orc = rel(got, refx), rel(ref64, refx)
    m_gpu, m_orc = elem_max(got, refx), elem_max(ref64, refx)
    bound = max(tol, e_orc)
    assert e_gpu <= bound, f"{what} FP64 relative L2 against the exact result {e_gpu:.3e} > {bound:.3e} (FP64 oracle {e_orc:.3e})"
    mb = ELEM_FACTOR * bound
    assert m_gpu <= mb, f"{what} FP64 per-element max against the exact result {m_gpu:.3e} > {mb:.3e} (FP64 oracle {m_orc:.3e})"
    return e_gpu, e_orc
