"""Element-wise parity metric shared by the GPU tests.

A whole-array relative L2 error can hide one misplaced bin under a small bar, so every parity
assertion uses parity_err: the larger of
  * the relative L2 error ||a - b|| / ||b||, and
  * the largest element error max |a - b| divided by MAXABS_FACTOR times the RMS of b.
`parity_err(a, b) <= tol` therefore holds the relative L2 error to tol and every element to
MAXABS_FACTOR * tol of the reference's RMS (a bin moved to its neighbour errs by about the RMS).
"""
import numpy as np

MAXABS_FACTOR = 20.0


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def max_abs_over_rms(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    rms = float(np.sqrt(np.mean(b * b))) if b.size else 0.0
    m = float(np.max(np.abs(a - b))) if b.size else 0.0
    return m / (rms if rms > 0 else 1.0)


def parity_err(a, b, factor: float = MAXABS_FACTOR) -> float:
    return max(rel_l2(a, b), max_abs_over_rms(a, b) / factor)
