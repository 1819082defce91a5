"""Python binding of the radiation-deposit library (the C ABI of include/rd.h).

Argument marshalling only: every step of the computation runs in the CUDA kernels of librd.so.
There is no fallback: if the library cannot be loaded, every call raises.

Low level: functions named exactly like the C entry points (rd_create_detector, ...) taking
ctypes structures / raw pointers and raising RDError on a non-zero status.
High level: RadiationDetector, which accepts torch tensors (CUDA or CPU) or numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from .build import LIB as _LIB_PATH
from .build import build as build_library

__all__ = [
    "RD_OK", "RD_ERR_ARG", "RD_ERR_CUDA", "RD_ERR_OOM", "RD_ERR_STATE", "RD_ERR_TIMEOUT",
    "RD_ERR_BOUNDS", "RD_ERR_INPUT", "RD_FP64", "RD_MIXED", "RD_NEAR", "RD_FAR", "RD_MEM_DEVICE",
    "RD_MEM_HOST", "RD_MEM_HOST_ASYNC", "RD_F32", "RD_F64", "RDError", "rd_detector_desc", "rd_traj", "rd_stats",
    "load_library", "library_path", "rd_create_detector", "rd_destroy", "rd_zero_fields",
    "rd_deposit_trajectories", "rd_read_fields", "rd_synchronize", "rd_get_stats",
    "rd_set_timing", "rd_adjoint_trajectories", "rd_set_adjoint_mode", "RD_ADJ_FP32", "RD_ADJ_COMPENSATED", "rd_shape", "rd_set_shape", "rd_get_shape",
    "rd_autotune_shape", "rd_deposit_batch", "rd_set_chunk", "rd_autotune",
    "rd_set_batch_budget", "rd_power_spectrum", "rd_deposit_stream", "rd_stream_reset",
    "rd_deposit_noalloc", "rd_measure_fma_peaks", "rd_check_bounded_wait", "rd_push_boris", "rd_last_error", "rd_version", "DepositFunction", "deposit_batch", "RadiationDetector", "build_library",
]

RD_OK, RD_ERR_ARG, RD_ERR_CUDA, RD_ERR_OOM, RD_ERR_STATE, RD_ERR_TIMEOUT, RD_ERR_BOUNDS, RD_ERR_INPUT = range(8)
RD_FP64, RD_MIXED = 0, 1
RD_NEAR, RD_FAR, RD_FARFIELD, RD_LINEAR, RD_HOLD_PREV, RD_QUADRATIC = 1, 2, 4, 8, 16, 32
RD_MEM_DEVICE, RD_MEM_HOST, RD_MEM_HOST_ASYNC = 0, 1, 2
RD_F32, RD_F64 = 0, 1
RD_SPEC_E, RD_SPEC_B = 0, 1
RD_ADJ_FP32, RD_ADJ_COMPENSATED = 0, 1

_STATUS = {0: "RD_OK", 1: "RD_ERR_ARG", 2: "RD_ERR_CUDA", 3: "RD_ERR_OOM", 4: "RD_ERR_STATE",
           5: "RD_ERR_TIMEOUT", 6: "RD_ERR_BOUNDS", 7: "RD_ERR_INPUT"}


class RDError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class rd_detector_desc(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int32), ("pix_pos", ctypes.c_void_p), ("pix_t0", ctypes.c_void_p),
                ("mem", ctypes.c_int32), ("t_min", ctypes.c_double), ("dt_det", ctypes.c_double),
                ("n_bins", ctypes.c_int32), ("precision", ctypes.c_int32), ("flags", ctypes.c_int32)]


class rd_traj(ctypes.Structure):
    _fields_ = [("n_part", ctypes.c_int32), ("n_samples", ctypes.c_int32), ("x", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("q", ctypes.c_void_p), ("mem", ctypes.c_int32),
                ("t0", ctypes.c_double), ("dt", ctypes.c_double)]


class rd_shape(ctypes.Structure):
    _fields_ = [("cells_per_cta", ctypes.c_int32), ("cells_per_thread", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("group", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class rd_stats(ctypes.Structure):
    _fields_ = [("n_clipped", ctypes.c_int64), ("n_deposits", ctypes.c_int64),
                ("n_bin_crossings", ctypes.c_int64), ("device_errors", ctypes.c_uint32), ("kernel_launches", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The shared library to load: RD_LIBRARY (a build of this source elsewhere) or the in-tree build."""
    return os.environ.get("RD_LIBRARY") or _LIB_PATH


def load_library(build_if_missing: bool = True):
    """Load librd.so (building it first if it is missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if build_if_missing and path == _LIB_PATH:
            build_library()
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        P, I = ctypes.c_void_p, ctypes.c_int32
        sig = {
            "rd_create_detector": ([ctypes.POINTER(rd_detector_desc), P, ctypes.POINTER(P)], I),
            "rd_destroy": ([P], I),
            "rd_zero_fields": ([P, P], I),
            "rd_deposit_trajectories": ([P, ctypes.POINTER(rd_traj), P], I),
            "rd_read_fields": ([P, P, P, I, I, P], I),
            "rd_write_fields": ([P, P, P, I, I, P], I),
            "rd_synchronize": ([P, P], I),
            "rd_get_stats": ([P, P, ctypes.POINTER(rd_stats)], I),
            "rd_set_timing": ([P, I], I),
            "rd_adjoint_trajectories": ([P, ctypes.POINTER(rd_traj), P, P, I, P, P, P], I),
            "rd_deposit_batch": ([I, ctypes.POINTER(P), ctypes.POINTER(rd_traj), P], I),
            "rd_set_chunk": ([P, I], I),
            "rd_set_adjoint_mode": ([P, I], I),
            "rd_set_shape": ([P, ctypes.POINTER(rd_shape)], I),
            "rd_get_shape": ([P, ctypes.POINTER(rd_shape)], I),
            "rd_autotune_shape": ([P, ctypes.POINTER(rd_traj), ctypes.c_char_p, P, ctypes.POINTER(rd_shape),
                                   ctypes.POINTER(I), ctypes.POINTER(ctypes.c_double)], I),
            "rd_set_batch_budget": ([P, ctypes.c_longlong], I),
            "rd_power_spectrum": ([P, I, P, P], I),
            "rd_deposit_stream": ([P, ctypes.POINTER(rd_traj), P], I),
            "rd_stream_reset": ([P], I),
            "rd_autotune": ([P, ctypes.POINTER(rd_traj), P, ctypes.POINTER(I)], I),
            "rd_deposit_noalloc": ([P, P, I, ctypes.c_double, ctypes.c_double, I, I, ctypes.POINTER(rd_traj), P,
                                    ctypes.POINTER(ctypes.c_uint32), P], I),
            "rd_measure_fma_peaks": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P], I),
            "rd_check_bounded_wait": ([I, P], I),
            "rd_push_boris": ([I, I, ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                               P, P, P, P, P], I),
            "rd_last_error": ([], ctypes.c_char_p),
            "rd_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != RD_OK:
        raise RDError(status, where, load_library().rd_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", stream)


# --------------------------------------------------------------------------------------------
# C entry points, one to one
# --------------------------------------------------------------------------------------------
def rd_create_detector(desc: rd_detector_desc, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load_library().rd_create_detector(ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(h)),
           "rd_create_detector")
    return h.value


def rd_destroy(det: int) -> None:
    _check(load_library().rd_destroy(det), "rd_destroy")


def rd_zero_fields(det: int, stream=None) -> None:
    _check(load_library().rd_zero_fields(det, _stream_ptr(stream)), "rd_zero_fields")


def rd_deposit_trajectories(det: int, traj: rd_traj, stream=None) -> None:
    _check(load_library().rd_deposit_trajectories(det, ctypes.byref(traj), _stream_ptr(stream)),
           "rd_deposit_trajectories")


def rd_read_fields(det: int, E_ptr, B_ptr, dtype: int, mem: int, stream=None) -> None:
    _check(load_library().rd_read_fields(det, E_ptr, B_ptr, dtype, mem, _stream_ptr(stream)),
           "rd_read_fields")


def rd_write_fields(det: int, E_ptr, B_ptr, dtype: int, mem: int, stream=None) -> None:
    _check(load_library().rd_write_fields(det, E_ptr, B_ptr, dtype, mem, _stream_ptr(stream)),
           "rd_write_fields")


def rd_synchronize(det: int, stream=None) -> None:
    _check(load_library().rd_synchronize(det, _stream_ptr(stream)), "rd_synchronize")


def rd_get_stats(det: int, stream=None) -> rd_stats:
    st = rd_stats()
    _check(load_library().rd_get_stats(det, _stream_ptr(stream), ctypes.byref(st)), "rd_get_stats")
    return st


def rd_adjoint_trajectories(det: int, traj: rd_traj, gE_ptr, gB_ptr, gdtype: int, gx_ptr, gu_ptr,
                            stream=None) -> None:
    _check(load_library().rd_adjoint_trajectories(det, ctypes.byref(traj), gE_ptr, gB_ptr, gdtype, gx_ptr,
                                                  gu_ptr, _stream_ptr(stream)), "rd_adjoint_trajectories")


def rd_deposit_batch(dets, trajs, stream=None) -> None:
    """dets: sequence of detector handles; trajs: sequence of rd_traj (device memory)."""
    n = len(dets)
    if n != len(trajs):
        raise ValueError("one trajectory set per detector")
    harr = (ctypes.c_void_p * n)(*dets)
    tarr = (rd_traj * n)(*trajs)
    _check(load_library().rd_deposit_batch(n, harr, tarr, _stream_ptr(stream)), "rd_deposit_batch")


def rd_set_chunk(det: int, chunk: int) -> None:
    _check(load_library().rd_set_chunk(det, int(chunk)), "rd_set_chunk")


def rd_set_shape(det: int, cells_per_cta: int = 256, cells_per_thread: int = 2, chunk: int = 0, group: int = 0) -> None:
    sh = rd_shape(int(cells_per_cta), int(cells_per_thread), int(chunk), int(group))
    _check(load_library().rd_set_shape(det, ctypes.byref(sh)), "rd_set_shape")


def rd_get_shape(det: int) -> dict:
    sh = rd_shape()
    _check(load_library().rd_get_shape(det, ctypes.byref(sh)), "rd_get_shape")
    return sh.as_dict()


def rd_autotune_shape(det: int, traj: rd_traj, cache_path=None, stream=None):
    """Tune the deposit shape for these trajectories; returns (shape dict, from_cache, ms)."""
    sh, hit, ms = rd_shape(), ctypes.c_int32(0), ctypes.c_double(0.0)
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(load_library().rd_autotune_shape(det, ctypes.byref(traj), path, _stream_ptr(stream), ctypes.byref(sh),
                                            ctypes.byref(hit), ctypes.byref(ms)), "rd_autotune_shape")
    return sh.as_dict(), bool(hit.value), float(ms.value)


def rd_set_adjoint_mode(det: int, mode: int) -> None:
    _check(load_library().rd_set_adjoint_mode(det, int(mode)), "rd_set_adjoint_mode")


def rd_set_batch_budget(det: int, nbytes: int) -> None:
    _check(load_library().rd_set_batch_budget(det, int(nbytes)), "rd_set_batch_budget")


def rd_deposit_stream(det: int, traj: rd_traj, stream=None) -> None:
    _check(load_library().rd_deposit_stream(det, ctypes.byref(traj), _stream_ptr(stream)), "rd_deposit_stream")


def rd_stream_reset(det: int) -> None:
    _check(load_library().rd_stream_reset(det), "rd_stream_reset")


def rd_power_spectrum(det: int, which: int, out_ptr: int, stream=None) -> None:
    _check(load_library().rd_power_spectrum(det, int(which), out_ptr, _stream_ptr(stream)), "rd_power_spectrum")


def rd_autotune(det: int, traj: rd_traj, stream=None) -> int:
    out = ctypes.c_int32(0)
    _check(load_library().rd_autotune(det, ctypes.byref(traj), _stream_ptr(stream), ctypes.byref(out)),
           "rd_autotune")
    return int(out.value)


def rd_deposit_noalloc(pix_pos_ptr, pix_t0_ptr, n_pix: int, t_min: float, dt_det: float, n_bins: int,
                       flags: int, traj: rd_traj, fields_ptr, want_errors: bool = True, stream=None):
    """Allocation-free deposit into caller-owned float[n_pix][n_bins][8] accumulators (device
    pointers throughout).  Returns the call's latched error bits when want_errors (synchronising)."""
    err = ctypes.c_uint32(0)
    _check(load_library().rd_deposit_noalloc(pix_pos_ptr, pix_t0_ptr, int(n_pix), float(t_min), float(dt_det),
                                             int(n_bins), int(flags), ctypes.byref(traj), fields_ptr,
                                             ctypes.byref(err) if want_errors else None, _stream_ptr(stream)),
           "rd_deposit_noalloc")
    return int(err.value) if want_errors else None


def rd_set_timing(det: int, enable: bool) -> None:
    _check(load_library().rd_set_timing(det, 1 if enable else 0), "rd_set_timing")


def rd_measure_fma_peaks(stream=None):
    """(FP32, FP64) fused multiply-add throughput of the current device in TFLOP/s, measured by
    the library's microbenchmark (diagnostic; one FMA = 2 flops)."""
    f32, f64 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    lib = load_library()
    _check(lib.rd_measure_fma_peaks(ctypes.byref(f32), ctypes.byref(f64), _stream_ptr(stream)), "rd_measure_fma_peaks")
    return f32.value, f64.value


def rd_push_boris(x, u, n_steps: int, dt: float, B, qm: float, x_out=None, u_out=None, stream=None):
    """Advance the charges with state x, u ([n_part][3] float64 CUDA tensors, updated in place) by
    n_steps Boris steps in the uniform field B; returns the new samples (x_out, u_out),
    [n_part][n_steps][3] CUDA tensors (allocated unless given)."""
    import torch
    for a in (x, u):
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous() and a.dim() == 2 and a.shape[1] == 3):
            raise ValueError("x and u must be contiguous float64 CUDA tensors [n_part][3]")
    n = x.shape[0]
    if x_out is None:
        x_out = torch.empty((n, n_steps, 3), dtype=torch.float64, device=x.device)
    if u_out is None:
        u_out = torch.empty((n, n_steps, 3), dtype=torch.float64, device=x.device)
    b = (ctypes.c_double * 3)(*[float(v) for v in B])
    _check(load_library().rd_push_boris(int(n), int(n_steps), float(dt), b, float(qm), x.data_ptr(), u.data_ptr(),
                                        x_out.data_ptr(), u_out.data_ptr(), _stream_ptr(stream)), "rd_push_boris")
    return x_out, u_out


def rd_check_bounded_wait(limit_ms: int = 20, stream=None) -> int:
    """Run the bounded-wait check (diagnostic); returns its status, RD_ERR_TIMEOUT when the wait ran
    out and was reported as the kernels report it (no exception for that expected outcome)."""
    return int(load_library().rd_check_bounded_wait(int(limit_ms), _stream_ptr(stream)))


def rd_last_error() -> str:
    return load_library().rd_last_error().decode(errors="replace")


def rd_version() -> str:
    return load_library().rd_version().decode()


# --------------------------------------------------------------------------------------------
# array marshalling
# --------------------------------------------------------------------------------------------
def _as_f64(a, keep):
    """(pointer, mem, n_elements) of an FP64 C-contiguous view of a torch tensor or array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            t = a.detach()
            if t.dtype != torch.float64 or not t.is_contiguous():
                t = t.to(torch.float64).contiguous()
            keep.append(t)
            return t.data_ptr(), (RD_MEM_DEVICE if t.is_cuda else RD_MEM_HOST), t.numel()
    except ImportError:
        pass
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    keep.append(arr)
    return arr.ctypes.data, RD_MEM_HOST, arr.size


class RadiationDetector:
    """A virtual detector on the GPU (see include/rd.h for the semantics).

    pix_pos [n_pix][3]; bin b of cell j covers [t_min + pix_t0[j] + b dt_det, ... + dt_det).
    precision: "mixed" (FP32 fields, FP64-accurate arrival times) or "fp64".
    """

    def __init__(self, pix_pos, t_min: float, dt_det: float, n_bins: int, pix_t0=None,
                 precision: str = "mixed", flags: int = RD_NEAR | RD_FAR, stream=None):
        keep = []
        pp, pmem, n = _as_f64(pix_pos, keep)
        if n % 3:
            raise ValueError("pix_pos must be [n_pix][3]")
        desc = rd_detector_desc()
        desc.n_pix = n // 3
        desc.pix_pos = pp
        desc.mem = pmem
        if pix_t0 is not None:
            tp, tmem, nt = _as_f64(pix_t0, keep)
            if nt != n // 3 or tmem != pmem:
                raise ValueError("pix_t0 must be [n_pix] in the same memory as pix_pos")
            desc.pix_t0 = tp
        desc.t_min = float(t_min)
        desc.dt_det = float(dt_det)
        desc.n_bins = int(n_bins)
        desc.precision = {"mixed": RD_MIXED, "fp64": RD_FP64}[precision]
        desc.flags = int(flags)
        self.n_pix, self.n_bins, self.precision = n // 3, int(n_bins), precision
        self.t_min, self.dt_det = float(t_min), float(dt_det)
        self._h = rd_create_detector(desc, stream)

    @classmethod
    def from_workload(cls, det, precision: str = "mixed", stream=None):
        return cls(det.pix_pos, det.t_min, det.dt_det, det.n_bins, det.pix_t0, precision, det.flags, stream)

    @property
    def handle(self) -> int:
        return self._h

    def traj_struct(self, x, u, q=None, t0: float = 0.0, dt: float = 1.0, keep=None):
        keep = [] if keep is None else keep
        xp, xmem, nx = _as_f64(x, keep)
        up, umem, nu = _as_f64(u, keep)
        shape = tuple(x.shape)
        if len(shape) != 3 or shape[2] != 3 or nx != nu or xmem != umem:
            raise ValueError("x and u must both be [n_part][n_samples][3] in the same memory")
        t = rd_traj()
        t.n_part, t.n_samples = shape[0], shape[1]
        t.x, t.u, t.mem = xp, up, xmem
        if q is not None:
            qp, qmem, nq = _as_f64(q, keep)
            if nq != shape[0] or qmem != xmem:
                raise ValueError("q must be [n_part] in the same memory as x")
            t.q = qp
        t.t0, t.dt = float(t0), float(dt)
        return t, keep

    def deposit(self, x, u, q=None, t0: float = 0.0, dt: float = 1.0, stream=None):
        """Accumulate the radiation of trajectories x, u ([n_part][n_samples][3])."""
        t, keep = self.traj_struct(x, u, q, t0, dt)
        rd_deposit_trajectories(self._h, t, stream)
        self._keep = keep      # inputs stay referenced until the next call

    def deposit_traj(self, tr, stream=None):
        self.deposit(tr.x, tr.u, tr.q, tr.t0, tr.dt, stream)

    def zero(self, stream=None):
        rd_zero_fields(self._h, stream)

    def read(self, dtype: str = "float64", device: str = "cpu", stream=None):
        """(E, B), each [n_pix][n_bins][3]; numpy on "cpu", torch tensors on "cuda"."""
        code = RD_F32 if dtype == "float32" else RD_F64
        if device == "cpu":
            E = np.empty((self.n_pix, self.n_bins, 3), dtype=np.float32 if code == RD_F32 else np.float64)
            B = np.empty_like(E)
            rd_read_fields(self._h, E.ctypes.data, B.ctypes.data, code, RD_MEM_HOST, stream)
            return E, B
        import torch
        tdt = torch.float32 if code == RD_F32 else torch.float64
        E = torch.empty((self.n_pix, self.n_bins, 3), dtype=tdt, device=device)
        B = torch.empty_like(E)
        rd_read_fields(self._h, E.data_ptr(), B.data_ptr(), code, RD_MEM_DEVICE, stream)
        return E, B

    def write(self, E, B, stream=None):
        """Set the fields to E, B ([n_pix][n_bins][3] each, float32 or float64; numpy arrays or CUDA
        tensors; None sets that part to zero): resumes a run checkpointed with read()."""
        arrs = [a for a in (E, B) if a is not None]
        if not arrs:
            rd_write_fields(self._h, None, None, RD_F64, RD_MEM_DEVICE, stream)
            return
        shape = (self.n_pix, self.n_bins, 3)
        if isinstance(arrs[0], np.ndarray):
            dt = np.float32 if arrs[0].dtype == np.float32 else np.float64
            E = None if E is None else np.ascontiguousarray(E, dtype=dt).reshape(shape)
            B = None if B is None else np.ascontiguousarray(B, dtype=dt).reshape(shape)
            code = RD_F32 if dt == np.float32 else RD_F64
            rd_write_fields(self._h, None if E is None else E.ctypes.data, None if B is None else B.ctypes.data,
                            code, RD_MEM_HOST, stream)
            return
        import torch
        tdt = torch.float32 if arrs[0].dtype == torch.float32 else torch.float64
        E = None if E is None else E.to(dtype=tdt).contiguous().reshape(shape)
        B = None if B is None else B.to(dtype=tdt).contiguous().reshape(shape)
        code = RD_F32 if tdt == torch.float32 else RD_F64
        rd_write_fields(self._h, None if E is None else E.data_ptr(), None if B is None else B.data_ptr(), code,
                        RD_MEM_DEVICE, stream)
        self._keep = (E, B)            # kept until the next call: the copy is asynchronous

    def deposit_stream(self, x, u, q=None, t0: float = 0.0, dt: float = 1.0, stream=None):
        """Deposit the next stretch of a streamed trajectory (new samples only, at t0 + k dt)."""
        t, keep = self.traj_struct(x, u, q, t0, dt)
        rd_deposit_stream(self._h, t, stream)
        self._keep = keep      # inputs stay referenced until the next call

    def stream_reset(self):
        rd_stream_reset(self._h)

    def power_spectrum(self, field: str = "E", stream=None):
        """dt_det^2 sum_c |FFT_b F_c[j][b]|^2 for k = 0..n_bins/2 (F = E or B): a float32 CUDA
        tensor [n_pix][n_bins/2 + 1]; angular frequency of column k is 2 pi k / (n_bins dt_det)."""
        import torch
        out = torch.empty((self.n_pix, self.n_bins // 2 + 1), dtype=torch.float32, device="cuda")
        rd_power_spectrum(self._h, RD_SPEC_B if field == "B" else RD_SPEC_E, out.data_ptr(), stream)
        return out

    def adjoint(self, x, u, q, t0, dt, gE, gB=None, stream=None):
        """d loss / d x and d loss / d u (FP64 CUDA tensors [n_part][n_samples][3]) for upstream
        gradients gE, gB ([n_pix][n_bins][3] CUDA tensors, float32 or float64; gB may be None)."""
        import torch
        t, keep = self.traj_struct(x, u, q, t0, dt)
        if t.mem != RD_MEM_DEVICE:
            raise ValueError("the adjoint needs CUDA trajectories")
        gdt = gE.dtype if gE is not None else gB.dtype
        code = RD_F32 if gdt == torch.float32 else RD_F64
        tdt = torch.float32 if code == RD_F32 else torch.float64
        gEc = None if gE is None else gE.detach().to(tdt).contiguous()
        gBc = None if gB is None else gB.detach().to(tdt).contiguous()
        for g in (gEc, gBc):
            if g is not None and (not g.is_cuda or g.numel() != self.n_pix * self.n_bins * 3):
                raise ValueError("seeds must be CUDA tensors of shape [n_pix][n_bins][3]")
        gx = torch.zeros(tuple(x.shape), dtype=torch.float64, device=x.device)
        gu = torch.zeros_like(gx)
        rd_adjoint_trajectories(self._h, t, None if gEc is None else gEc.data_ptr(),
                                None if gBc is None else gBc.data_ptr(), code, gx.data_ptr(), gu.data_ptr(),
                                stream)
        self._keep = keep + [gEc, gBc]
        return gx, gu

    def set_chunk(self, chunk: int):
        rd_set_chunk(self._h, chunk)

    def set_shape(self, cells_per_cta: int = 256, cells_per_thread: int = 2, chunk: int = 0, group: int = 0):
        rd_set_shape(self._h, cells_per_cta, cells_per_thread, chunk, group)

    def shape(self) -> dict:
        return rd_get_shape(self._h)

    def autotune_shape(self, x, u, q=None, t0: float = 0.0, dt: float = 1.0, cache_path=None, stream=None):
        """Tune (or take from the JSON cache at cache_path) the deposit shape for these trajectories;
        returns (shape dict, from_cache, ms).  Fields are zeroed afterwards."""
        t, keep = self.traj_struct(x, u, q, t0, dt)
        out = rd_autotune_shape(self._h, t, cache_path, stream)
        del keep
        return out

    def set_adjoint_mode(self, mode):
        """RD_ADJ_FP32 / "fp32" (default) or RD_ADJ_COMPENSATED / "compensated" (RD_MIXED only)."""
        if isinstance(mode, str):
            mode = {"fp32": RD_ADJ_FP32, "compensated": RD_ADJ_COMPENSATED}[mode]
        rd_set_adjoint_mode(self._h, mode)

    def set_batch_budget(self, nbytes: int):
        """Bytes of per-sample records per launch group of batches led by this detector (0 = 4 GiB)."""
        rd_set_batch_budget(self._h, nbytes)

    def autotune(self, x, u, q=None, t0: float = 0.0, dt: float = 1.0, stream=None) -> int:
        """Pick the fastest step chunk for these trajectories (fields are zeroed afterwards)."""
        t, keep = self.traj_struct(x, u, q, t0, dt)
        chunk = rd_autotune(self._h, t, stream)
        del keep
        return chunk

    def synchronize(self, stream=None):
        rd_synchronize(self._h, stream)

    def stats(self, stream=None) -> rd_stats:
        return rd_get_stats(self._h, stream)

    def set_timing(self, enable: bool = True):
        rd_set_timing(self._h, enable)

    def close(self):
        if getattr(self, "_h", None):
            rd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def deposit_batch(detectors, trajectories, stream=None):
    """One persistent launch depositing trajectories[i] = (x, u, q, t0, dt) (CUDA tensors) into
    detectors[i] (RadiationDetector, mixed precision) for all i."""
    keep, trajs = [], []
    for det, (x, u, q, t0, dt) in zip(detectors, trajectories):
        t, k = det.traj_struct(x, u, q, t0, dt)
        keep.extend(k)
        trajs.append(t)
    rd_deposit_batch([d.handle for d in detectors], trajs, stream)
    return keep


class DepositFunction:
    """Differentiable deposit: (x, u) -> (E, B) through a RadiationDetector (mixed or FP64).

    forward: zero the detector, deposit, return E, B as float64 CUDA tensors [n_pix][n_bins][3];
    backward: the adjoint kernel gives d loss / d x and d loss / d u.  q, t0 and dt are constants.
    Usage: E, B = DepositFunction.apply(det, x, u, q, t0, dt)."""

    _fn = None

    @classmethod
    def apply(cls, det, x, u, q, t0, dt):
        if cls._fn is None:
            import torch

            class _Deposit(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, u, det, q, t0, dt):
                    det.zero()
                    det.deposit(x.detach(), u.detach(), q, t0, dt)
                    E, B = det.read("float64", x.device)
                    ctx.det, ctx.q, ctx.t0, ctx.dt = det, q, t0, dt
                    ctx.save_for_backward(x, u)
                    return E, B

                @staticmethod
                def backward(ctx, gE, gB):
                    x, u = ctx.saved_tensors
                    gx, gu = ctx.det.adjoint(x.detach(), u.detach(), ctx.q, ctx.t0, ctx.dt, gE, gB)
                    return gx.to(x.dtype), gu.to(u.dtype), None, None, None, None

            cls._fn = _Deposit
        return cls._fn.apply(x, u, det, q, t0, dt)
