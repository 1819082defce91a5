"""The C ABI library builds, loads and exports every entry point include/rd.h declares.

No GPU is needed: only argument checks that fail before any CUDA call are exercised.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2302_14812_gb300 as rd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"RD_API\s+[\w\s\*]+?\b(rd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = rd.build_library()
    return ctypes.CDLL(path)


def test_header_is_plain_c():
    subprocess.run(["gcc", "-fsyntax-only", "-Wall", "-Werror", "-x", "c", "-std=c99", HEADER], check=True)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 8
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_entry_point():
    for n in declared_functions():
        assert hasattr(rd, n), n


def test_argument_errors_without_gpu():
    lib = rd.load_library()
    assert rd.rd_version().startswith("rd ")
    # NULL detector / descriptor are rejected before any CUDA call
    assert lib.rd_create_detector(None, None, None) == rd.RD_ERR_ARG
    assert "NULL" in rd.rd_last_error()
    assert lib.rd_zero_fields(None, None) == rd.RD_ERR_ARG
    assert lib.rd_deposit_trajectories(None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_read_fields(None, None, None, 0, 0, None) == rd.RD_ERR_ARG
    assert lib.rd_write_fields(None, None, None, rd.RD_F32, rd.RD_MEM_HOST, None) == rd.RD_ERR_ARG
    assert lib.rd_destroy(None) == rd.RD_OK
    d = rd.rd_detector_desc()
    d.n_pix = 0
    h = ctypes.c_void_p()
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    d.n_pix, d.n_bins, d.dt_det = 4, 8, -1.0
    buf = (ctypes.c_double * 12)()
    d.pix_pos = ctypes.cast(buf, ctypes.c_void_p)
    d.mem = rd.RD_MEM_HOST
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    d.dt_det, d.precision = 0.1, 7
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    with pytest.raises(rd.RDError) as ei:
        rd.rd_create_detector(d)
    assert ei.value.status == rd.RD_ERR_ARG
    # an RD_MIXED detector holds at most 2^22 bins per cell (walk offsets stay in int32)
    d.precision, d.n_bins = rd.RD_MIXED, (1 << 22) + 1
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    assert "4194304" in rd.rd_last_error()
    # the far-field limit keeps only the radiation term
    d.n_bins, d.flags = 8, rd.RD_NEAR | rd.RD_FARFIELD
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    assert "RD_FARFIELD" in rd.rd_last_error()
    d.flags = 8
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    # the two interpolation variants are alternatives; unknown bits are refused
    d.flags = rd.RD_NEAR | rd.RD_FAR | rd.RD_LINEAR | rd.RD_HOLD_PREV
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    assert "alternatives" in rd.rd_last_error()
    d.flags = rd.RD_NEAR | 64
    assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
    for both in (rd.RD_LINEAR | rd.RD_QUADRATIC, rd.RD_HOLD_PREV | rd.RD_QUADRATIC):
        d.flags = rd.RD_NEAR | rd.RD_FAR | both
        assert lib.rd_create_detector(ctypes.byref(d), None, ctypes.byref(h)) == rd.RD_ERR_ARG
        assert "alternatives" in rd.rd_last_error()
    assert lib.rd_set_batch_budget(None, 0) == rd.RD_ERR_ARG
    assert lib.rd_deposit_stream(None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_stream_reset(None) == rd.RD_ERR_ARG
    assert lib.rd_set_chunk(None, 0) == rd.RD_ERR_ARG
    # the other entry points refuse bad arguments before any CUDA call
    assert lib.rd_synchronize(None, None) == rd.RD_ERR_ARG
    assert lib.rd_get_stats(None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_set_timing(None, 1) == rd.RD_ERR_ARG
    assert lib.rd_adjoint_trajectories(None, None, None, None, 0, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_deposit_batch(0, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_autotune(None, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_power_spectrum(None, 0, None, None) == rd.RD_ERR_ARG
    assert lib.rd_check_bounded_wait(0, None) == rd.RD_ERR_ARG
    assert lib.rd_check_bounded_wait(2001, None) == rd.RD_ERR_ARG
    B = (ctypes.c_double * 3)(0.0, 0.0, 1.0)
    assert lib.rd_push_boris(-1, 1, 0.1, B, 1.0, None, None, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_push_boris(1, 1, 0.1, None, 1.0, None, None, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_push_boris(1, 1, 0.1, B, 1.0, None, None, None, None, None) == rd.RD_ERR_ARG
    B[2] = float("nan")
    assert lib.rd_push_boris(1, 1, 0.1, B, 1.0, None, None, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_push_boris(0, 5, 0.1, (ctypes.c_double * 3)(), 1.0, None, None, None, None, None) == rd.RD_OK
    # rd_deposit_noalloc: one particle's records must fit the 56 MiB record area (917500 samples)
    t = rd.rd_traj()
    t.n_part, t.n_samples, t.mem, t.t0, t.dt = 1, 917501, rd.RD_MEM_DEVICE, 0.0, 0.1
    t.x = t.u = 16                                    # never dereferenced: the size check comes first
    cells = (ctypes.c_double * 3)()
    assert lib.rd_deposit_noalloc(ctypes.cast(cells, ctypes.c_void_p), None, 1, 0.0, 0.1, 8, 0, ctypes.byref(t),
                                  16, None, None) == rd.RD_ERR_ARG
    assert "917500" in rd.rd_last_error()
    t.mem = rd.RD_MEM_HOST
    assert lib.rd_deposit_noalloc(ctypes.cast(cells, ctypes.c_void_p), None, 1, 0.0, 0.1, 8, 0, ctypes.byref(t),
                                  16, None, None) == rd.RD_ERR_ARG
    assert "device trajectories" in rd.rd_last_error()
    # rd_deposit_noalloc checks flags as rd_create_detector does: a set that selects no term of
    # Eq. 1 (the far-field limit or an interpolation variant alone) is refused before any CUDA call
    t.mem = rd.RD_MEM_DEVICE
    t.n_samples = 10
    for flags in (rd.RD_FARFIELD, rd.RD_LINEAR, rd.RD_HOLD_PREV, rd.RD_QUADRATIC, rd.RD_NEAR | rd.RD_FARFIELD, rd.RD_NEAR | 64,
                  rd.RD_NEAR | rd.RD_LINEAR | rd.RD_HOLD_PREV):
        assert lib.rd_deposit_noalloc(ctypes.cast(cells, ctypes.c_void_p), None, 1, 0.0, 0.1, 8, flags,
                                      ctypes.byref(t), 16, None, None) == rd.RD_ERR_ARG, flags
    assert "Eq. 1" in (lib.rd_deposit_noalloc(ctypes.cast(cells, ctypes.c_void_p), None, 1, 0.0, 0.1, 8,
                                              rd.RD_LINEAR, ctypes.byref(t), 16, None, None) and rd.rd_last_error())


def test_shape_entry_points_refuse_bad_arguments():
    lib = rd.load_library()
    sh = rd.rd_shape(256, 2, 0, 0)
    assert lib.rd_set_shape(None, ctypes.byref(sh)) == rd.RD_ERR_ARG
    assert lib.rd_get_shape(None, ctypes.byref(sh)) == rd.RD_ERR_ARG
    assert lib.rd_autotune_shape(None, None, None, None, None, None, None) == rd.RD_ERR_ARG
    assert lib.rd_set_adjoint_mode(None, 1) == rd.RD_ERR_ARG
