"""Power spectra of the detector's time series (rd_power_spectrum) on the GPU.

The oracle of a spectrum is numpy's FFT of the fields (a library routine), taken of the GPU
detector's own fields (checks the FFT) and of the oracle's fields (checks deposit + FFT end to
end).  The Section 4 benchmark at its full size (512 cells x 131072 bins) is then compared with
Eq. 8 and Eq. 9 exactly as the oracle pins do at 33 cells.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rd.load_library()
    oracle.build()


def numpy_power(F, dt_det):
    """dt_det^2 sum_c |rfft(F_c)|^2, F: [n_pix][n_bins][3]."""
    return dt_det ** 2 * np.sum(np.abs(np.fft.rfft(F, axis=1)) ** 2, axis=2)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_power_spectrum_equals_fft_of_fields(precision):
    """Random smooth motions, 300 cells (ragged cell blocks), 1024 bins: the GPU spectrum of E and
    of B against numpy's FFT of the same detector's fields (FP32 FFT: 1e-5)."""
    import torch
    rng = np.random.default_rng(5)
    tr = W.random_smooth(4, 500, 0.02, max_u=2.0, seed=5)
    pos = rng.normal(size=(300, 3)) * 20.0
    det = W.Detector(pos, rng.uniform(-1, 1, 300), 10.0, 0.021, 1024)
    d = rd.RadiationDetector.from_workload(det, precision)
    d.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
              tr.t0, tr.dt)
    E, B = d.read()
    for field, F in (("E", E), ("B", B)):
        P = d.power_spectrum(field).cpu().numpy()
        assert P.shape == (det.n_pix, det.n_bins // 2 + 1)
        assert parity_err(P, numpy_power(F, det.dt_det)) <= 1e-5
    d.close()


@pytest.mark.parametrize("n_bins", [2, 8192, 16384])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_power_spectrum_lengths(n_bins, precision):
    """The shortest series, the longest transformed in shared memory (8192) and the shortest
    transformed by passes over the whole batch (16384), against numpy's FFT of the same fields."""
    import torch
    rng = np.random.default_rng(n_bins)
    tr = W.random_smooth(2, 300, 0.02, max_u=2.0, seed=9)
    pos = rng.normal(size=(37, 3)) * 15.0
    dt_det = 8.0 / n_bins
    det = W.Detector(pos, None, 10.0, dt_det, n_bins)
    d = rd.RadiationDetector.from_workload(det, precision)
    d.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
              tr.t0, tr.dt)
    E, B = d.read()
    assert np.any(E != 0.0)
    for field, F in (("E", E), ("B", B)):
        P = d.power_spectrum(field).cpu().numpy()
        assert P.shape == (det.n_pix, n_bins // 2 + 1)
        assert parity_err(P, numpy_power(F, det.dt_det)) <= 1e-5
    d.close()


def test_power_spectrum_needs_power_of_two_bins():
    det = W.Detector(np.array([[10.0, 0.0, 0.0]]), None, 0.0, 0.1, 1000)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    with pytest.raises(rd.RDError) as ei:
        d.power_spectrum()
    assert ei.value.status == rd.RD_ERR_ARG
    d.close()


def test_section4_benchmark_full_size_spectra():
    """The paper's benchmark (gamma 50, K 10, 512 cells x 131072 bins): the mixed deposit and GPU
    spectrum against the oracle + numpy FFT on 8 cells (1e-4), then Eq. 9 for the line-integrated
    spectrum (3 %, w/w_c in [0.15, 2.2]) and Eq. 8 on axis (8 %, w/w_c in [0.1, 2.2])."""
    import torch
    from test_oracle_pins import _eq8_shape
    sp = pytest.importorskip("scipy.special")
    si = pytest.importorskip("scipy.integrate")
    gam, K = 50.0, 10.0
    tr, det, th = W.config_sinusoidal_benchmark(n_cells=512)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    d.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
              tr.t0, tr.dt)
    P = d.power_spectrum("E").double().cpu().numpy()
    assert d.stats().n_clipped == 0
    d.close()
    sel = np.linspace(0, 511, 8).astype(np.int32)
    Eo, _, _ = oracle.deposit(tr, det, sel)
    assert parity_err(P[sel], numpy_power(Eo, det.dt_det)) <= 1e-4

    _, wb = W.undulator_params(gam, K, 2.0 * math.pi / 0.1)
    wc = 1.5 * K * gam ** 2 * wb
    w = 2.0 * math.pi * np.arange(det.n_bins // 2 + 1) / (det.n_bins * det.dt_det)
    P = P / np.sinc(w * det.dt_det / (2.0 * math.pi))[None, :] ** 2
    edges = np.geomspace(0.02, 3.0, 25) * wc
    mid = np.sqrt(edges[1:] * edges[:-1])
    band = np.stack([P[:, (w >= a) & (w < b)].mean(axis=1) for a, b in zip(edges[:-1], edges[1:])], axis=1)

    def F(x):
        return x * si.quad(lambda v: sp.kv(5.0 / 3.0, v), x, np.inf)[0]
    tint = band.sum(axis=0)
    eq9 = np.array([np.mean([F(x / wc) for x in np.linspace(a, b, 8)]) for a, b in zip(edges[:-1], edges[1:])])
    ref = int(np.argmax(tint))
    r9 = (tint / tint[ref]) / (eq9 / eq9[ref])
    use9 = (mid >= 0.15 * wc) & (mid <= 2.2 * wc)
    assert np.all(np.abs(r9[use9] - 1.0) < 0.03), r9[use9]

    c0 = int(np.argmin(np.abs(th)))
    t8 = np.array([np.mean(_eq8_shape(np.linspace(a, b, 16), th[c0], gam, K, wb))
                   for a, b in zip(edges[:-1], edges[1:])])
    ref = int(np.argmax(band[c0]))
    r8 = (band[c0] / band[c0, ref]) / (t8 / t8[ref])
    use8 = (mid >= 0.1 * wc) & (mid <= 2.2 * wc)
    assert np.all(np.abs(r8[use8] - 1.0) < 0.08), r8[use8]
