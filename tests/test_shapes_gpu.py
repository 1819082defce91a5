"""Deposit shapes of the mixed kernel (cells per CTA x cells per thread, step chunk, work-order
group) and the shape autotuner with its JSON cache.

Every compiled shape runs the same per-(cell, interval) arithmetic; only the order in which FP32
partial sums reach a bin and, with another chunk, the placement of the FP64 arrival anchors
differ.  Bars: the oracle's mixed bar (1e-4, every element within 2e-3 of its size or the RMS)
and, against the default shape, 2e-6 (same chunk) or 2e-5 (another chunk).
"""
import json

import numpy as np
import pytest

import oracle
import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err

pytestmark = pytest.mark.gpu

SHAPES = [(256, 2), (128, 2), (64, 2), (256, 1), (128, 1), (64, 1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rd.load_library()
    oracle.build()


def _dev(tr):
    import torch
    return (torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(), tr.t0, tr.dt)


def _deposit(tr, det, shape=None):
    d = rd.RadiationDetector.from_workload(det, "mixed")
    if shape is not None:
        d.set_shape(*shape)
    d.deposit(*_dev(tr))
    E, B = d.read()
    st = d.stats()
    d.close()
    return E, B, st


def _ragged():
    rng = np.random.default_rng(5)
    tr = W.random_smooth(5, 333, 0.02, max_u=3.0, seed=5)
    pos = rng.normal(size=(300, 3)) * 20.0
    pos += 25.0 * pos / np.linalg.norm(pos, axis=1, keepdims=True)
    return tr, W.Detector(pos, rng.uniform(-1.0, 1.0, 300), 30.0, 0.013, 700)


def _multi_edge():
    tr = W.oscillator_ensemble(4, 700, amp_range=(0.5, 1.0), seed=11)
    rng = np.random.default_rng(11)
    n = 300
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    pos = np.stack([50.0 * sgn, rng.uniform(-5, 5, n), rng.uniform(-5, 5, n)], axis=1)
    shift = np.where(np.arange(n) < 150, 0.0, np.where(np.arange(n) % 4 < 2, 20.0, -20.0))
    return tr, W.Detector(pos, shift, 30.0, 1.2 * tr.dt, 1000)


@pytest.mark.parametrize("case", ["ragged", "multi_edge"])
@pytest.mark.parametrize("shape", SHAPES)
def test_every_shape_matches_the_oracle(shape, case):
    """300 cells (ragged last block for every cells-per-CTA), per-cell time origins, windows that cut
    arrivals (clip tracking) and, in the second case, intervals passing two or more bin edges (the
    exact re-walk of a tile): every shape against the oracle and against the default shape."""
    tr, det = _ragged() if case == "ragged" else _multi_edge()
    E, B, st = _deposit(tr, det, shape)
    Eo, Bo, clipped = oracle.deposit(tr, det)
    assert parity_err(E, Eo) <= 1e-4 and parity_err(B, Bo) <= 1e-4
    E0, B0, st0 = _deposit(tr, det)
    assert parity_err(E, E0) <= 2e-6 and parity_err(B, B0) <= 2e-6
    assert st.n_clipped == st0.n_clipped and st.device_errors == 0


def test_shape_chunk_and_group():
    """Explicit chunks (anchors every 64 or 100 intervals) and groups (1, 3, 8 cell blocks, one group
    ragged) give the default result to the chunk's rounding."""
    tr, det = W.config_undulator(n_part=6, n_steps=1500, n_side=24, n_bins=512, seed=3)
    E0, B0, _ = _deposit(tr, det)
    Eo, Bo, _ = oracle.deposit(tr, det, np.arange(0, det.n_pix, 37, dtype=np.int32))
    for shape in ((256, 2, 64, 1), (128, 1, 100, 3), (64, 2, 0, 8), (256, 2, 1500, 2)):
        E, B, _ = _deposit(tr, det, shape)
        assert parity_err(E, E0) <= 2e-5 and parity_err(B, B0) <= 2e-5, shape
        assert parity_err(E[::37], Eo) <= 1e-4, shape


def test_unsupported_shape_is_refused():
    det = W.Detector(W.spherical_cap(2, 10.0, 0.3), None, 8.0, 0.05, 64)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    for bad in ((96, 2), (256, 4), (256, 2, -1, 0), (256, 2, 0, -2)):
        with pytest.raises(rd.RDError) as ei:
            d.set_shape(*bad)
        assert ei.value.status == rd.RD_ERR_ARG
    assert d.shape() == {"cells_per_cta": 256, "cells_per_thread": 2, "chunk": 0, "group": 0}
    d.close()
    d = rd.RadiationDetector.from_workload(det, "fp64")
    with pytest.raises(rd.RDError) as ei:
        d.set_shape(128, 2)
    assert ei.value.status == rd.RD_ERR_STATE
    d.close()


def test_autotuner_times_caches_and_reuses(tmp_path):
    """The autotuner picks a compiled shape, writes it to the JSON cache, and a second tuner on the same
    problem takes it from the cache without timing; the tuned deposit matches the oracle; a far-field
    detector keeps the default cells per CTA and per thread; a malformed cache is reported."""
    tr, det = W.config_undulator(n_part=8, n_steps=1200, n_side=20, n_bins=512, seed=4)
    cache = tmp_path / "shapes.json"
    d = rd.RadiationDetector.from_workload(det, "mixed")
    x, u, q, t0, dt = _dev(tr)
    shape, hit, ms = d.autotune_shape(x, u, q, t0, dt, cache_path=str(cache))
    assert not hit and ms > 0.0
    assert (shape["cells_per_cta"], shape["cells_per_thread"]) in SHAPES
    assert d.shape() == shape
    E, _ = d.read()
    assert not np.any(E)                                  # fields zeroed after the trials
    doc = json.loads(cache.read_text())
    assert doc["rd_shape_cache"] == 1 and len(doc["entries"]) == 1
    entry = next(iter(doc["entries"].values()))
    assert entry["cells_per_cta"] == shape["cells_per_cta"] and entry["chunk"] == shape["chunk"]
    d.deposit(x, u, q, t0, dt)
    E, B = d.read()
    sel = np.arange(0, det.n_pix, 29, dtype=np.int32)
    Eo, Bo, _ = oracle.deposit(tr, det, sel)
    assert parity_err(E[sel], Eo) <= 1e-4 and parity_err(B[sel], Bo) <= 1e-4
    d.close()
    d2 = rd.RadiationDetector.from_workload(det, "mixed")
    shape2, hit2, ms2 = d2.autotune_shape(x, u, q, t0, dt, cache_path=str(cache))
    assert hit2 and shape2 == shape and ms2 == pytest.approx(ms, rel=1e-5)
    d2.close()
    det_ff = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins, W.RD_FAR | W.RD_FARFIELD)
    d3 = rd.RadiationDetector.from_workload(det_ff, "mixed")
    shape3, hit3, _ = d3.autotune_shape(x, u, q, t0, dt, cache_path=str(cache))
    assert not hit3 and (shape3["cells_per_cta"], shape3["cells_per_thread"]) == (256, 2)
    assert len(json.loads(cache.read_text())["entries"]) == 2
    d3.close()
    bad = tmp_path / "bad.json"
    bad.write_text("{\"rd_shape_cache\": 1, \"entries\": {\"k\": ")
    d4 = rd.RadiationDetector.from_workload(det, "mixed")
    with pytest.raises(rd.RDError) as ei:
        d4.autotune_shape(x, u, q, t0, dt, cache_path=str(bad))
    assert ei.value.status == rd.RD_ERR_ARG and "malformed" in str(ei.value)
    d4.close()


def test_batch_uses_each_detectors_chunk_and_group():
    """Problems with tuned (chunk, group) in one batched launch equal their separate deposits."""
    import torch
    probs = [W.config_undulator(n_part=5, n_steps=900, n_side=16, n_bins=256, seed=1),
             W.config_undulator(n_part=3, n_steps=700, n_side=12, n_bins=300, gamma=8.0, seed=2)]
    dets = [rd.RadiationDetector.from_workload(det, "mixed") for _, det in probs]
    dets[0].set_shape(256, 2, 128, 1)
    dets[1].set_shape(256, 2, 700, 0)
    sep = []
    for (tr, det), d in zip(probs, dets):
        s = rd.RadiationDetector.from_workload(det, "mixed")
        s.set_shape(*d.shape().values())
        s.deposit(*_dev(tr))
        sep.append(s.read())
        s.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        keep = rd.deposit_batch(dets, [_dev(tr) for tr, _ in probs], stream)
        out = [d.read(stream=stream) for d in dets]
    del keep
    for (E, B), (Es, Bs) in zip(out, sep):
        assert parity_err(E, Es) <= 2e-6 and parity_err(B, Bs) <= 2e-6
    for d in dets:
        d.close()
