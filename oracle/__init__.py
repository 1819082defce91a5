"""FP64 CPU oracle of the RaDiO deposit (ctypes wrapper around rd_oracle.c).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's CPU baseline
are the only users.  The product path (the CUDA library and its binding) never imports this
package, and the two share no code.

Parity of each function:
  field, beta, arrival_time, bin_coord, deposit_interval, deposit_interval_lin, deposit_interval_quad,
  deposit (all flag variants)                                       -- pinned by tests/test_oracle_*.py
  deposit_dir (complex-step derivative)                            -- pinned by central finite differences
  deposit_ext (long double evaluation of deposit)                   -- pinned against deposit where FP64 rounding
                                                                      is negligible, and against the rounding
                                                                      bound of Eq. 2 where it is not
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librd_oracle.so")
_SRC = [os.path.join(_HERE, "rd_oracle.c"), os.path.join(_HERE, "rd_oracle_core.h")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rd_oracle.c into oracle/_build/librd_oracle.so (gcc, no fused multiply-add)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", tmp, _SRC[0], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int32), ("pix_pos", ctypes.c_void_p), ("pix_t0", ctypes.c_void_p),
                ("t_min", ctypes.c_double), ("dt_det", ctypes.c_double), ("n_bins", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("n_part", ctypes.c_int32), ("n_samples", ctypes.c_int32),
                ("x", ctypes.c_void_p), ("u", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("t0", ctypes.c_double), ("dt", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            lib.rdo_field.argtypes = [D, D, D, D, ctypes.c_double, ctypes.c_int32, D, D]
            lib.rdo_field.restype = None
            lib.rdo_arrival_time.argtypes = [ctypes.c_double, D, D]
            lib.rdo_arrival_time.restype = ctypes.c_double
            lib.rdo_bin_coord.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_double, D, D,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int32]
            lib.rdo_bin_coord.restype = ctypes.c_double
            lib.rdo_deposit_interval.argtypes = [ctypes.c_double, ctypes.c_double, D, ctypes.c_int32, D]
            lib.rdo_deposit_interval.restype = ctypes.c_int32
            lib.rdo_deposit_interval_lin.argtypes = [ctypes.c_double, ctypes.c_double, D, D, ctypes.c_int32, D]
            lib.rdo_deposit_interval_lin.restype = ctypes.c_int32
            lib.rdo_deposit_interval_quad.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, D, D, D,
                                                      ctypes.c_int32, D]
            lib.rdo_deposit_interval_quad.restype = ctypes.c_int32
            lib.rdo_beta.argtypes = [D, D]
            lib.rdo_beta.restype = None
            lib.rdo_deposit.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.c_int32, D, D,
                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
            lib.rdo_deposit.restype = ctypes.c_int32
            lib.rdo_deposit_ext.argtypes = lib.rdo_deposit.argtypes
            lib.rdo_deposit_ext.restype = ctypes.c_int32
            lib.rdo_deposit_dir.argtypes = [ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_double, D, D, ctypes.c_int32]
            lib.rdo_deposit_dir.restype = ctypes.c_int32
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))


class OracleError(RuntimeError):
    pass


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def field(x, beta, bdot, P, q=1.0, flags=3):
    """Eq. 1 at one sample: returns (E[3], B[3])."""
    lib = _load()
    xs, bs, ds, ps = _vec(x), _vec(beta), _vec(bdot), _vec(P)
    E = np.zeros(3)
    B = np.zeros(3)
    lib.rdo_field(_dp(xs), _dp(bs), _dp(ds), _dp(ps), float(q), int(flags), _dp(E), _dp(B))
    return E, B


def beta(u):
    lib = _load()
    us = _vec(u)
    b = np.zeros(3)
    lib.rdo_beta(_dp(us), _dp(b))
    return b


def arrival_time(t, x, P) -> float:
    """Eq. 2: t + |x - P| (c = 1)."""
    lib = _load()
    return float(lib.rdo_arrival_time(float(t), _dp(_vec(x)), _dp(_vec(P))))


def bin_coord(t0, k, dt, x, P, T0, inv_dt_det, flags=3) -> float:
    """Arrival time of sample k at cell P in bin units: Eq. 2, or Eq. 3 when flags has bit 4."""
    lib = _load()
    return float(lib.rdo_bin_coord(float(t0), int(k), float(dt), _dp(_vec(x)), _dp(_vec(P)),
                                   float(T0), float(inv_dt_det), int(flags)))


def deposit_interval(a, c, F, n_bins, row=None):
    """Deposit the constant 6-vector F over [a, c] (bin units) into row[n_bins][6]."""
    lib = _load()
    if row is None:
        row = np.zeros((n_bins, 6))
    Fs = _vec(F)
    clipped = lib.rdo_deposit_interval(float(a), float(c), _dp(Fs), int(n_bins), _dp(row))
    return row, int(clipped)


def deposit_interval_lin(a, c, F0, F1, n_bins, row=None):
    """Deposit the field going linearly from F0 at a to F1 at c (bin units) into row[n_bins][6]."""
    lib = _load()
    if row is None:
        row = np.zeros((n_bins, 6))
    clipped = lib.rdo_deposit_interval_lin(float(a), float(c), _dp(_vec(F0)), _dp(_vec(F1)), int(n_bins), _dp(row))
    return row, int(clipped)


def deposit_interval_quad(p, a, c, Fp, Fa, Fc, n_bins, row=None):
    """Deposit over [a, c] the quadratic through (p, Fp), (a, Fa), (c, Fc) (bin units) into row[n_bins][6]."""
    lib = _load()
    if row is None:
        row = np.zeros((n_bins, 6))
    clipped = lib.rdo_deposit_interval_quad(float(p), float(a), float(c), _dp(_vec(Fp)), _dp(_vec(Fa)),
                                            _dp(_vec(Fc)), int(n_bins), _dp(row))
    return row, int(clipped)


def _problem(tr, det, keep):
    x = np.ascontiguousarray(tr.x, dtype=np.float64)
    u = np.ascontiguousarray(tr.u, dtype=np.float64)
    q = np.ascontiguousarray(tr.q, dtype=np.float64)
    pos = np.ascontiguousarray(det.pix_pos, dtype=np.float64)
    t0a = None if det.pix_t0 is None else np.ascontiguousarray(det.pix_t0, dtype=np.float64)
    keep.extend([x, u, q, pos, t0a])
    pr = _Problem()
    pr.n_pix = int(pos.shape[0])
    pr.pix_pos = pos.ctypes.data
    pr.pix_t0 = None if t0a is None else t0a.ctypes.data
    pr.t_min = float(det.t_min)
    pr.dt_det = float(det.dt_det)
    pr.n_bins = int(det.n_bins)
    pr.flags = int(det.flags)
    pr.n_part = int(x.shape[0])
    pr.n_samples = int(x.shape[1])
    pr.x = x.ctypes.data
    pr.u = u.ctypes.data
    pr.q = q.ctypes.data
    pr.t0 = float(tr.t0)
    pr.dt = float(tr.dt)
    return pr


def _selection(det, sel, keep):
    if sel is None:
        return None, det.n_pix
    s = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
    keep.append(s)
    return s.ctypes.data, int(s.size)


def deposit(tr, det, sel=None, n_threads=None):
    """Oracle detector rows for the selected cells: (E[n_sel][n_bins][3], B[...], n_clipped)."""
    lib = _load()
    keep = []
    pr = _problem(tr, det, keep)
    sp, n_sel = _selection(det, sel, keep)
    E = np.zeros((n_sel, det.n_bins, 3))
    B = np.zeros((n_sel, det.n_bins, 3))
    clipped = ctypes.c_int64(0)
    st = lib.rdo_deposit(ctypes.byref(pr), sp, n_sel, _dp(E), _dp(B),
                         int(n_threads or default_threads()), ctypes.byref(clipped))
    if st != 0:
        raise OracleError({1: "bad arguments", 2: "invalid trajectory (chord speed >= 1 or not finite)",
                           3: "out of memory"}.get(st, f"status {st}"))
    return E, B, int(clipped.value)


def deposit_ext(tr, det, sel=None, n_threads=None):
    """deposit() evaluated in long double (same formulas, longer mantissa): measures the rounding
    of the FP64 evaluation, chiefly Eq. 2's t + R where R is large and a step's arrival increment
    dt (1 - beta.n) is small."""
    lib = _load()
    keep = []
    pr = _problem(tr, det, keep)
    sp, n_sel = _selection(det, sel, keep)
    E = np.zeros((n_sel, det.n_bins, 3))
    B = np.zeros((n_sel, det.n_bins, 3))
    clipped = ctypes.c_int64(0)
    st = lib.rdo_deposit_ext(ctypes.byref(pr), sp, n_sel, _dp(E), _dp(B),
                             int(n_threads or default_threads()), ctypes.byref(clipped))
    if st != 0:
        raise OracleError(f"rdo_deposit_ext status {st}")
    return E, B, int(clipped.value)


def deposit_dir(tr, det, p, k, which, comp, h=1e-20, sel=None, n_threads=None):
    """Exact derivative (complex step) of particle p's detector contribution with respect to
    x[p][k][comp] (which='x') or u[p][k][comp] (which='u'): (dE, dB) for the selected cells."""
    lib = _load()
    keep = []
    pr = _problem(tr, det, keep)
    sp, n_sel = _selection(det, sel, keep)
    dE = np.zeros((n_sel, det.n_bins, 3))
    dB = np.zeros((n_sel, det.n_bins, 3))
    w = {"x": 0, "u": 1}[which] if isinstance(which, str) else int(which)
    st = lib.rdo_deposit_dir(ctypes.byref(pr), sp, n_sel, int(p), int(k), w, int(comp), float(h),
                             _dp(dE), _dp(dB), int(n_threads or default_threads()))
    if st != 0:
        raise OracleError(f"rdo_deposit_dir status {st}")
    return dE, dB
