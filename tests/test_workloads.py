"""Input generators (no method arithmetic): shapes, seeding, and the device-side generator of the
plasma-mirror ensemble against the host one."""
import math

import numpy as np
import pytest

from paper_2302_14812_gb300 import workloads as W


def test_plasma_mirror_device_generator_matches_host_generator():
    """The PyTorch generator (used for ensembles too large to build on the host) gives the host
    generator's trajectories for the same particle slice, to rounding."""
    torch = pytest.importorskip("torch")
    sl = slice(100, 130)
    tr = W.plasma_mirror_surface(n_steps=1000, particles=sl)
    x, u, q, (t0, dt) = W.plasma_mirror_surface_torch(sl, n_steps=1000, device="cpu", sub=7)
    assert x.dtype == torch.float64 and tuple(x.shape) == tr.x.shape
    assert np.abs(x.numpy() - tr.x).max() <= 1e-13 * np.abs(tr.x).max()
    assert np.abs(u.numpy() - tr.u).max() <= 1e-13 * np.abs(tr.u).max()
    assert t0 == tr.t0 and dt == tr.dt and np.array_equal(q.numpy(), tr.q)


def test_plasma_mirror_ensemble_is_subluminal_and_seeded():
    tr = W.plasma_mirror_surface(n_part=2000, n_steps=400, particles=slice(0, 40))
    v = np.linalg.norm(np.diff(tr.x, axis=1), axis=-1) / tr.dt
    assert v.max() < 1.0
    tr2 = W.plasma_mirror_surface(n_part=2000, n_steps=400, particles=slice(20, 40))
    assert np.array_equal(tr.x[20:], tr2.x)          # a slice is the same particles


def test_plasma_mirror_detector_window_covers_arrivals():
    """pix_t0 = |x_pix| - reach and 4096 bins of 5 dt: every arrival of the surface electrons
    lies inside the window of every cell (on a sample of cells and particles)."""
    tr = W.plasma_mirror_surface(n_part=100_000, n_steps=10_000, particles=slice(0, 3))
    det = W.plasma_mirror_detector(tr.dt, n_side=16)
    k = np.arange(tr.n_samples)
    for p in range(tr.n_part):
        R = np.linalg.norm(det.pix_pos[:, None, :] - tr.x[p][None], axis=-1)
        ub = (tr.t0 + k[None] * tr.dt + R - (det.t_min + det.pix_t0[:, None])) / det.dt_det
        assert ub.min() > 0.0 and ub.max() < det.n_bins
    assert math.isclose(det.dt_det, 5.0 * tr.dt)


def test_boris_generator_rotation_closed_form():
    """The numpy Boris generator: in a uniform field |u| is kept and u turns about B by exactly
    2 atan(|t|) per step, t = (qm dt/2) |B| / gamma (the Boris rotation); chords stay below c."""
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=(5, 3))
    x0 = rng.normal(size=(5, 3))
    B, qm, dt, n = np.array([0.3, -0.4, 1.2]), 2.0, 0.03, 500
    tr = W.boris_uniform_field(x0, u0, n, dt, B, qm)
    assert np.max(np.abs(np.linalg.norm(tr.u, axis=2) - np.linalg.norm(u0, axis=1)[:, None])) < 1e-12
    bh = B / np.linalg.norm(B)
    perp = tr.u - np.sum(tr.u * bh, axis=2, keepdims=True) * bh
    e1 = perp[:, 0] / np.linalg.norm(perp[:, 0], axis=1, keepdims=True)
    e2 = np.cross(bh, e1)
    ang = np.unwrap(np.arctan2(np.sum(perp * e2[:, None], axis=2), np.sum(perp * e1[:, None], axis=2)), axis=1)
    g = np.sqrt(1.0 + np.sum(u0 * u0, axis=1))
    phi = 2.0 * np.arctan(0.5 * qm * dt * np.linalg.norm(B) / g)
    assert np.max(np.abs(np.abs(ang[:, -1]) - n * phi)) < 1e-10
    chord = np.linalg.norm(np.diff(tr.x, axis=1), axis=2) / dt
    assert chord.max() < 1.0


def test_batch_problems_torch_matches_numpy_generator():
    """The device generator of the 64-problem set (PyTorch FP64, run here on the CPU) reproduces the
    numpy generator: same kinds, sizes, detectors and time axes, trajectories equal to rounding."""
    torch = pytest.importorskip("torch")
    ref = W.batch_problems(64, seed=4, scale=0.002)
    dev = W.batch_problems_torch(64, seed=4, scale=0.002, device="cpu")
    assert len(ref) == len(dev) == 64
    kinds = set()
    for (k1, tr, det), (k2, (x, u, q, t0, dt), det2) in zip(ref, dev):
        kinds.add(k1)
        assert k1 == k2 and x.shape == tr.x.shape and u.shape == tr.u.shape
        assert dt == tr.dt and t0 == tr.t0
        assert det.n_bins == det2.n_bins and det.t_min == det2.t_min and det.dt_det == det2.dt_det
        assert np.array_equal(det.pix_pos, det2.pix_pos)
        scale = max(1.0, float(np.max(np.abs(tr.x))))
        assert np.max(np.abs(x.numpy() - tr.x)) <= 1e-12 * scale
        assert np.max(np.abs(u.numpy() - tr.u)) <= 1e-13 * max(1.0, float(np.max(np.abs(tr.u))))
        assert np.array_equal(q.numpy(), tr.q)
    assert kinds == {"undulator", "circular", "oscillator"}
