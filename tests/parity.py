"""Element-wise parity metric shared by the GPU tests.

A whole-array relative L2 error can hide one misplaced bin under a small bar, so every parity
assertion uses parity_err: the larger of
  * the relative L2 error ||a - b|| / ||b||, and
  * the largest element error |a_i - b_i| divided by MAXABS_FACTOR times max(|b_i|, RMS of b).
`parity_err(a, b) <= tol` therefore holds the relative L2 error to tol and every element to
MAXABS_FACTOR * tol of its own size, or of the reference's RMS where the element is smaller than
that (a bin moved to its neighbour, or a value where the reference is near zero, errs by about the
RMS or the element itself; pulsed signals, whose peak bins are far above the RMS, keep a relative
bar on those bins).
"""
import numpy as np

MAXABS_FACTOR = 20.0


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def max_elem_err(a, b) -> float:
    """max_i |a_i - b_i| / max(|b_i|, RMS of b)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    rms = float(np.sqrt(np.mean(b * b)))
    scale = np.maximum(np.abs(b), rms if rms > 0 else 1.0)
    return float(np.max(np.abs(a - b) / scale))


def parity_err(a, b, factor: float = MAXABS_FACTOR) -> float:
    return max(rel_l2(a, b), max_elem_err(a, b) / factor)
