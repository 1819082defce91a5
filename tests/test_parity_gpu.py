"""GPU deposit (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative L2 over every compared element, E and B separately):
  FP64 path  1e-10   (both sides evaluate the arrival time with the same FP64 operations, so bin
                      weights agree; differences come from field arithmetic order, ~1e-15)
  mixed path 1e-4    (FP32 field and accumulation, FP64-accurate arrival time)
"""
import math

import numpy as np
import pytest

import oracle
import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rd.load_library()
    oracle.build()


def gpu_run(tr, det, precision, where="device", calls=None):
    import torch
    d = rd.RadiationDetector.from_workload(det, precision)
    parts = calls or [tr]
    for t in parts:
        if where == "device":
            d.deposit(torch.from_numpy(t.x).cuda(), torch.from_numpy(t.u).cuda(),
                      torch.from_numpy(t.q).cuda(), t.t0, t.dt)
        else:
            d.deposit(t.x, t.u, t.q, t.t0, t.dt)
    E, B = d.read("float64", "cpu")
    st = d.stats()
    d.close()
    return E, B, st


def check(tr, det, precision, sel=None, where="device", Eo=None, Bo=None, clip_exact=None):
    E, B, st = gpu_run(tr, det, precision, where)
    if Eo is None:
        Eo, Bo, clipped = oracle.deposit(tr, det, sel)
    else:
        clipped = None
    if sel is not None:
        E, B = E[sel], B[sel]
    eE, eB = parity_err(E, Eo), parity_err(B, Bo)
    assert np.abs(Eo).max() > 0
    assert eE <= TOL[precision] and eB <= TOL[precision], (precision, eE, eB)
    if clip_exact is None:
        clip_exact = precision == "fp64" and sel is None
    if clip_exact and clipped is not None:
        assert st.n_clipped == clipped
    return eE, eB


# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_circular_orbit_full(precision):
    """One electron on a circular orbit (gamma 5, 2000 steps), 64-cell arc at 1e3, 1024 bins."""
    tr, det = W.config_circular()
    check(tr, det, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_ensembles_ragged(precision, seed):
    """Random smooth motions, 300 cells (two cell blocks, ragged), 333 intervals (several
    64-sample tiles and chunks with a ragged tail), per-cell time origins and a window that cuts
    some arrivals (clipped counts must match the oracle exactly in FP64)."""
    rng = np.random.default_rng(seed)
    tr = W.random_smooth(7, 333, 0.02, max_u=3.0, seed=seed)
    pos = rng.normal(size=(300, 3)) * 20.0
    pos += 25.0 * pos / np.linalg.norm(pos, axis=1, keepdims=True)
    t0 = rng.uniform(-1.0, 1.0, 300)
    det = W.Detector(pos, t0, 30.0, 0.013, 700)
    check(tr, det, precision)


def _multi_edge_case():
    """Relativistic oscillators along x seen from +-x at distance 50 with bins 1.2 dt wide: about 8 %
    of the (cell, interval) pairs pass two or more bin edges, mixed with single crossings in every
    64-interval tile.  Cells 0-255 see every arrival inside the window with a margin (no clip
    tracking); cells 256-511 have time origins shifted by +-20 so the window cuts their arrivals at
    one end or the other (clip tracking)."""
    tr = W.oscillator_ensemble(6, 900, amp_range=(0.5, 1.0), seed=11)
    rng = np.random.default_rng(11)
    n = 512
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    pos = np.stack([50.0 * sgn, rng.uniform(-5, 5, n), rng.uniform(-5, 5, n)], axis=1)
    shift = np.where(np.arange(n) < 256, 0.0, np.where(np.arange(n) % 4 < 2, 20.0, -20.0))
    return tr, W.Detector(pos, shift, 30.0, 1.2 * tr.dt, 1161)


def _bin_coords(tr, det):
    k = np.arange(tr.n_samples)
    tt = tr.t0 + k * tr.dt
    T0 = det.t_min + (0.0 if det.pix_t0 is None else det.pix_t0)
    return np.array([(tt[None] + np.linalg.norm(det.pix_pos[:, None, :] - tr.x[p][None], axis=-1)
                      - np.asarray(T0).reshape(-1, 1)) / det.dt_det for p in range(tr.n_part)])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_intervals_spanning_several_bins(precision):
    """Intervals that pass two or more bin edges (the mixed kernel's fast walk stops such a cell
    and walks its tile again with the exact step) among ordinary ones, in tracked and untracked
    cell blocks; every cell against the oracle."""
    tr, det = _multi_edge_case()
    u = _bin_coords(tr, det)
    edges = np.diff(np.floor(u), axis=-1)
    frac = float(np.mean(edges >= 2))
    assert 0.02 < frac < 0.5, frac
    assert u[:, :256].min() >= 1.0 and u[:, :256].max() <= det.n_bins - 1.0     # untracked block
    assert u[:, 256:].min() < 0.0 and u[:, 256:].max() > det.n_bins              # window cuts block 2
    check(tr, det, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_undulator_small(precision):
    """Undulator ensemble (gamma 20, K 1, 4000 steps), 8 electrons, 32x32 cap, 2048 bins."""
    tr, det = W.config_undulator(n_part=8, n_side=32)
    check(tr, det, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_undulator_full_size_sampled_cells(precision):
    """The benchmark workload at full size (1000 electrons x 4000 steps x 128x128 cells x 2048
    bins), launched as the benchmark launches it; the oracle computes 6 sampled cells."""
    tr, det = W.config_undulator()
    sel = np.array([0, 127, 64 * 128 + 64, 5000, 128 * 127, 128 * 128 - 1], dtype=np.int32)
    check(tr, det, precision, sel=sel)


@pytest.mark.parametrize("mode", ["linear", "hold_prev", "quadratic", "farfield"])
def test_variants_full_size_sampled_cells(mode):
    """The interpolation variants and the far-field limit on the benchmark workload at full size:
    the mixed path deposits the whole 128x128 x 2048 detector as the benchmark launches it, the
    FP64 path a detector of the 6 sampled cells; both against the oracle on those cells."""
    import torch
    tr, det = W.config_undulator()
    det.flags = {"linear": W.RD_NEAR | W.RD_FAR | W.RD_LINEAR,
                 "hold_prev": W.RD_NEAR | W.RD_FAR | W.RD_HOLD_PREV,
                 "quadratic": W.RD_NEAR | W.RD_FAR | W.RD_QUADRATIC,
                 "farfield": W.RD_FAR | W.RD_FARFIELD}[mode]
    sel = np.array([0, 127, 64 * 128 + 64, 5000, 128 * 127, 128 * 128 - 1], dtype=np.int32)
    Eo, Bo, _ = oracle.deposit(tr, det, sel)
    assert np.abs(Eo).max() > 0
    x, u, q = (torch.from_numpy(a).cuda() for a in (tr.x, tr.u, tr.q))
    d = rd.RadiationDetector.from_workload(det, "mixed")
    d.deposit(x, u, q, tr.t0, tr.dt)
    E, B = d.read("float32", "cuda")
    st = d.stats()
    d.close()
    idx = torch.from_numpy(sel.astype(np.int64)).cuda()
    E, B = E[idx].double().cpu().numpy(), B[idx].double().cpu().numpy()
    assert st.device_errors == 0
    assert parity_err(E, Eo) <= TOL["mixed"] and parity_err(B, Bo) <= TOL["mixed"], mode
    d64 = rd.RadiationDetector.from_workload(det.subset(sel), "fp64")
    d64.deposit(x, u, q, tr.t0, tr.dt)
    E64, B64 = d64.read()
    d64.close()
    assert parity_err(E64, Eo) <= TOL["fp64"] and parity_err(B64, Bo) <= TOL["fp64"], mode


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plasma_mirror_reduced(precision):
    """Plasma-mirror-like surface (a0 5, 20 harmonics, 10000 steps), 300 electrons, 48x48 plane
    with per-cell time origins; the oracle computes 8 cells spread over the plane."""
    tr, det = W.config_plasma_mirror(n_part=300, n_side=48, particles=slice(0, 300))
    sel = np.array([0, 47, 24 * 48 + 24, 1000, 1500, 2000, 48 * 47, 48 * 48 - 1], dtype=np.int32)
    check(tr, det, precision, sel=sel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_helical_section_3_3_full_size(precision):
    """The Section 3.3 example at its size: one electron on a helix (gamma 57.3, K 0.8, dt 0.1,
    400 steps), 64x64 spherical detector over 0.1 rad around the axis at R = 1e6, 8192 bins of
    1.33e-5 (118 bins per radiation period on the axis), per-cell time origins.  The oracle
    computes 8 cells from the centre to the corners."""
    tr, det = W.config_helical()
    sel = np.array([0, 63, 31 * 64 + 31, 32 * 64 + 32, 31 * 64 + 40, 2000, 64 * 63, 64 * 64 - 1], dtype=np.int32)
    check(tr, det, precision, sel=sel)


@pytest.mark.parametrize("gamma", [300.0, 1000.0])
def test_high_gamma_against_extended_precision(gamma):
    """Undulator electrons at gamma 300 and 1000 (R = 1e4, 16x16 cap over +-1.5/gamma, 2048 bins).
    Here Eq. 2 in FP64 rounds t + R to ulp(R) while a step's arrival increment is dt (1 - beta.n)
    ~ 1e-9, so the reference is the oracle evaluated in long double.  Both forms stay within the
    mixed bar of it (measured: FP64 4e-7 / 1.2e-5, mixed 5.7e-6 / 4.5e-5), and the FP64 form still
    agrees with the FP64 oracle to the FP64 bar at gamma 300."""
    tr, det = W.config_undulator(n_part=4, n_steps=2000, n_side=16, n_bins=2048, gamma=gamma, K=1.0,
                                 distance=1e4)
    sel = np.array([0, 7, 8 * 16 + 8, 100, 255], dtype=np.int32)
    Ee, Be, _ = oracle.deposit_ext(tr, det, sel)
    got = {}
    for precision in ("fp64", "mixed"):
        E, B, _ = gpu_run(tr, det, precision)
        got[precision] = (E[sel], B[sel])
        assert parity_err(E[sel], Ee) <= 1e-4 and parity_err(B[sel], Be) <= 1e-4, precision
    if gamma <= 300.0:
        E64, B64, _ = oracle.deposit(tr, det, sel)
        E, B = got["fp64"]
        assert parity_err(E, E64) <= TOL["fp64"] and parity_err(B, B64) <= TOL["fp64"]


def _config_sample(name):
    """(trajectories, detector, cell sample) of one workload configuration, at its full detector
    geometry and step count with few particles."""
    rng = np.random.default_rng(41)
    if name == "circular":                       # synchrotron arc, all 64 cells
        tr, det = W.config_circular()
        return tr, det, np.arange(det.n_pix, dtype=np.int32)
    if name == "undulator":                      # the headline geometry, 16 electrons
        tr, det = W.config_undulator(n_part=16)
    elif name == "plasma_mirror":                # full plane and steps, 40 of the electrons
        tr, det = W.config_plasma_mirror(n_part=100_000, particles=slice(0, 40))
    elif name == "batch":                        # one problem of each kind from the 64-problem set
        probs = W.batch_problems(64, seed=4, scale=0.002)
        kind, tr, det = next(p for p in probs if p[0] == "oscillator")
    else:                                        # the adjoint workload's geometry
        tr, det = W.config_undulator(n_part=16, n_steps=2000, n_side=64, n_bins=1024, gamma=10.0, K=1.0,
                                     n_periods=10.0, distance=1e4, seed=5)
    sel = np.sort(rng.choice(det.n_pix, 6, replace=False)).astype(np.int32)
    return tr, det, sel


@pytest.mark.parametrize("name", ["circular", "undulator", "plasma_mirror", "batch", "adjoint"])
def test_every_config_against_extended_precision(name):
    """Each workload configuration on a cell sample against the oracle evaluated in long double,
    which does not share the FP64 rounding of Eq. 2 that the FP64 kernel and the FP64 oracle both
    fix (reading A17): the FP64 form within 1e-7 (the spread FP64 rounding of t + R leaves at these
    distances is ~1e-9), the mixed form within its 1e-4 bar."""
    tr, det, sel = _config_sample(name)
    Ee, Be, _ = oracle.deposit_ext(tr, det, sel)
    assert np.abs(Ee).max() > 0
    sub = det.subset(sel)
    for precision, bar in (("fp64", 1e-7), ("mixed", 1e-4)):
        E, B, st = gpu_run(tr, sub, precision)
        assert st.device_errors == 0
        eE, eB = parity_err(E, Ee), parity_err(B, Be)
        print(f"{name} {precision} vs long double: E {eE:.2e} B {eB:.2e}")
        assert eE <= bar and eB <= bar, (name, precision, eE, eB)
    if name == "batch":
        probs = [p for p in W.batch_problems(64, seed=4, scale=0.002) if p[0] != "oscillator"]
        for kind in ("undulator", "circular"):
            _, tr, det = next(p for p in probs if p[0] == kind)
            sel = np.array([0, det.n_pix // 2, det.n_pix - 1], dtype=np.int32)
            Ee, Be, _ = oracle.deposit_ext(tr, det, sel)
            E, B, _ = gpu_run(tr, det.subset(sel), "fp64")
            assert parity_err(E, Ee) <= 1e-7 and parity_err(B, Be) <= 1e-7, kind


# --------------------------------------------------------------------------------------------
# edge cases and API behaviour
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_memory_inputs(precision):
    tr = W.random_smooth(3, 150, 0.03, seed=4)
    det = W.Detector(W.spherical_cap(5, 20.0, 0.6), None, 16.0, 0.02, 600)
    check(tr, det, precision, where="host")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_chunks_and_particle_chunks_accumulate(precision):
    """Deposits accumulate: particle subsets and step chunks sharing one sample sum to the whole
    (the run-time mode of Section 3.1)."""
    tr = W.random_smooth(4, 200, 0.03, seed=5)
    det = W.Detector(W.spherical_cap(4, 18.0, 0.5), None, 14.0, 0.017, 900)
    Eo, Bo, _ = oracle.deposit(tr, det)
    parts = [tr.subset([0, 1]).steps(0, 77), tr.subset([0, 1]).steps(77, 200), tr.subset([2, 3])]
    E, B, _ = gpu_run(tr, det, precision, calls=parts)
    assert parity_err(E, Eo) <= TOL[precision] and parity_err(B, Bo) <= TOL[precision]


def test_empty_and_degenerate_inputs():
    import torch
    det = W.Detector(W.spherical_cap(2, 10.0, 0.3), None, 8.0, 0.05, 64)
    for precision in ("fp64", "mixed"):
        d = rd.RadiationDetector.from_workload(det, precision)
        d.deposit(np.zeros((0, 5, 3)), np.zeros((0, 5, 3)), np.zeros(0), 0.0, 0.1)   # no particle
        d.deposit(np.zeros((2, 1, 3)), np.zeros((2, 1, 3)), np.ones(2), 0.0, 0.1)    # no interval
        E, B = d.read()
        assert np.all(E == 0) and np.all(B == 0)
        # a single interval
        tr = W.random_smooth(1, 1, 0.05, seed=3)
        d.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), None, tr.t0, tr.dt)
        E, B = d.read()
        Eo, Bo, _ = oracle.deposit(W.Trajectories(tr.x, tr.u, np.ones(1), tr.t0, tr.dt), det)
        assert parity_err(E, Eo) <= TOL[precision]
        d.zero()
        E, _ = d.read()
        assert np.all(E == 0)
        d.close()


def test_mixed_maximum_bins_per_cell():
    """RD_MIXED at its largest row (2^22 bins) with a full 256-cell block, so that field offsets
    (row * n_bins + bin) reach 2^30 - 1.  Every cell's arrivals lie in the last few thousand bins;
    for odd cells they run past the window's end (clipped there).  Intervals span 1-15 bins (the
    exact re-walk handles them).  Cells at both ends of both halves of the block against the
    oracle; device-side readback (the detector holds 34 GB)."""
    import torch
    n_bins = 1 << 22
    tr = W.random_smooth(2, 200, 0.02, max_u=2.0, seed=21)
    pos = W.spherical_cap(16, 12.0, 0.6)
    t = tr.t0 + tr.dt * np.arange(tr.n_samples)
    arr = t[None, None, :] + np.linalg.norm(pos[:, None, None, :] - tr.x[None], axis=-1)
    dt_det = 2.5e-3
    first = np.where(np.arange(pos.shape[0]) % 2 == 0, n_bins - 3500, n_bins - 1500)
    det = W.Detector(pos, arr.min(axis=(1, 2)) - first * dt_det, 0.0, dt_det, n_bins)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    d.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
              tr.t0, tr.dt)
    assert d.stats().n_clipped > 0
    E, B = d.read("float32", "cuda")
    sel = np.array([0, 1, 127, 128, 254, 255], dtype=np.int32)
    Eg = E[torch.from_numpy(sel).long().cuda()].double().cpu().numpy()
    Bg = B[torch.from_numpy(sel).long().cuda()].double().cpu().numpy()
    del E, B
    d.close()
    Eo, Bo, _ = oracle.deposit(tr, det, sel)
    assert np.any(Eo[:, -1] != 0.0)                   # odd cells reach the last bin
    assert parity_err(Eg, Eo) <= TOL["mixed"] and parity_err(Bg, Bo) <= TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_window_entirely_missed_counts_clipped(precision):
    tr = W.random_smooth(2, 90, 0.03, seed=8)
    det = W.Detector(W.spherical_cap(3, 20.0, 0.5), None, 1e4, 0.01, 100)
    E, B, st = gpu_run(tr, det, precision)
    assert np.all(E == 0) and np.all(B == 0)
    assert st.n_clipped == 2 * 90 * 9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_near_and_far_terms(precision):
    tr = W.random_smooth(2, 120, 0.03, seed=9)
    for flags in (W.RD_NEAR, W.RD_FAR):
        det = W.Detector(W.spherical_cap(3, 15.0, 0.5), None, 11.0, 0.02, 800, flags=flags)
        check(tr, det, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_superluminal_chord_rejected(precision):
    tr = W.random_smooth(1, 20, 0.05, seed=1)
    tr.x[0, 7] = tr.x[0, 6] + np.array([0.06, 0.0, 0.0])
    det = W.Detector(np.array([[10.0, 0, 0]]), None, 0.0, 0.1, 100)
    d = rd.RadiationDetector.from_workload(det, precision)
    d.deposit(tr.x, tr.u, tr.q, tr.t0, tr.dt)
    with pytest.raises(rd.RDError) as ei:
        d.read()
    assert ei.value.status == rd.RD_ERR_INPUT
    d.close()


def test_read_fields_device_and_f32():
    import torch
    tr = W.random_smooth(2, 60, 0.03, seed=10)
    det = W.Detector(W.spherical_cap(3, 12.0, 0.5), None, 9.0, 0.02, 300)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    d.deposit_traj(tr)
    E64, B64 = d.read("float64", "cpu")
    E32, B32 = d.read("float32", "cpu")
    Ed, Bd = d.read("float32", "cuda")
    torch.cuda.synchronize()
    assert np.array_equal(E32, E64.astype(np.float32))
    assert np.array_equal(Ed.cpu().numpy(), E32) and np.array_equal(Bd.cpu().numpy(), B32)
    # asynchronous readback into page-locked host memory, on a side stream
    s = torch.cuda.Stream()
    Ea = torch.empty((det.n_pix, det.n_bins, 3), dtype=torch.float32).pin_memory()
    Ba = torch.empty_like(Ea).pin_memory()
    rd.rd_read_fields(d.handle, Ea.data_ptr(), Ba.data_ptr(), rd.RD_F32, rd.RD_MEM_HOST_ASYNC, s)
    d.synchronize(s)
    assert np.array_equal(Ea.numpy(), E32) and np.array_equal(Ba.numpy(), B32)
    d.close()


# --------------------------------------------------------------------------------------------
# far-field limit (RD_FARFIELD): Eq. 3 arrival times, radiation term at the cell's (n_c, R_c)
# --------------------------------------------------------------------------------------------
def _farfield_cases():
    rng = np.random.default_rng(8)
    tr1 = W.random_smooth(5, 333, 0.02, max_u=3.0, seed=8)
    pos = rng.normal(size=(300, 3)) * 20.0
    pos += 25.0 * pos / np.linalg.norm(pos, axis=1, keepdims=True)
    det1 = W.Detector(pos, rng.uniform(-1.0, 1.0, 300), 30.0, 0.013, 700, flags=W.RD_FAR | W.RD_FARFIELD)
    tr2, det2 = W.config_undulator(n_part=6, n_side=24, n_bins=1024, seed=4)
    det2.flags = W.RD_FAR | W.RD_FARFIELD
    tr3, det3 = _multi_edge_case()
    det3.flags = W.RD_FAR | W.RD_FARFIELD
    return [(tr1, det1), (tr2, det2), (tr3, det3)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_farfield_limit(precision, case):
    """Random motions with per-cell origins and window cuts; the undulator ensemble on a cap at
    1e4; intervals spanning several bins in tracked and untracked blocks: every cell against
    the oracle's far-field limit (clipped counts exact in FP64)."""
    tr, det = _farfield_cases()[case]
    check(tr, det, precision)


def test_farfield_flag_checks():
    import torch
    det = W.Detector(np.array([[10.0, 0.0, 0.0]]), None, 0.0, 0.1, 64, flags=W.RD_NEAR | W.RD_FARFIELD)
    with pytest.raises(rd.RDError) as ei:
        rd.RadiationDetector.from_workload(det, "mixed")
    assert ei.value.status == rd.RD_ERR_ARG
    det.flags = W.RD_FAR | W.RD_FARFIELD
    d = rd.RadiationDetector.from_workload(det, "mixed")
    tr = W.random_smooth(1, 20, 0.05, seed=1)
    x, u = torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda()
    with pytest.raises(rd.RDError) as ei:
        d.adjoint(x, u, None, tr.t0, tr.dt, torch.zeros((1, 64, 3), dtype=torch.float32, device="cuda"))
    assert ei.value.status == rd.RD_ERR_STATE
    d.close()


# --------------------------------------------------------------------------------------------
# linear-in-time interpolation (RD_LINEAR), alone and with the far-field limit
# --------------------------------------------------------------------------------------------
def _linear_cases():
    out = []
    for tr, det in _farfield_cases():               # same inputs as the far-field cases
        det.flags = W.RD_NEAR | W.RD_FAR | W.RD_LINEAR
        out.append((tr, det))
    tr, det = _farfield_cases()[1]
    det.flags = W.RD_FAR | W.RD_FARFIELD | W.RD_LINEAR
    out.append((tr, det))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_linear_interpolation(precision, case):
    """Window cuts and per-cell origins; the undulator ensemble; intervals spanning several bins
    in tracked and untracked blocks; the undulator in the far-field limit: every cell against the
    oracle's linear interpolation (clipped counts exact in FP64)."""
    tr, det = _linear_cases()[case]
    check(tr, det, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_hold_previous_field(precision, case):
    """RD_HOLD_PREV (interval k holds the field of sample k-1) on the same four cases as the linear
    interpolation, every cell against the oracle."""
    tr, det = _linear_cases()[case]
    det.flags = (det.flags & ~W.RD_LINEAR) | W.RD_HOLD_PREV
    check(tr, det, precision)


def test_hold_previous_streamed_and_batched():
    """RD_HOLD_PREV through rd_deposit_stream (stretches of 1, 7, 64 and the rest) and through one
    batched launch with a held-current problem beside it: the same fields as one plain call."""
    import torch
    tr, det = _linear_cases()[0]
    det.flags = W.RD_NEAR | W.RD_FAR | W.RD_HOLD_PREV
    ref = rd.RadiationDetector.from_workload(det, "mixed")
    xd, ud, qd = (torch.from_numpy(a).cuda() for a in (tr.x, tr.u, tr.q))
    ref.deposit(xd, ud, qd, tr.t0, tr.dt)
    Er, Br = ref.read()
    d = rd.RadiationDetector.from_workload(det, "mixed")
    k = 0
    for m in (1, 7, 64, tr.n_samples):
        b = min(tr.n_samples, k + m)
        d.deposit_stream(xd[:, k:b].contiguous(), ud[:, k:b].contiguous(), qd, tr.t0 + k * tr.dt, tr.dt)
        k = b
        if k >= tr.n_samples:
            break
    E, B = d.read()
    assert parity_err(E, Er) <= 2e-6 and parity_err(B, Br) <= 2e-6
    d.close()
    det_held = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins, W.RD_NEAR | W.RD_FAR)
    dets = [rd.RadiationDetector.from_workload(det, "mixed"), rd.RadiationDetector.from_workload(det_held, "mixed")]
    keep = rd.deposit_batch(dets, [(xd, ud, qd, tr.t0, tr.dt)] * 2)
    E0, B0 = dets[0].read()
    assert parity_err(E0, Er) <= 2e-6 and parity_err(B0, Br) <= 2e-6
    Eh, _, _ = oracle.deposit(tr, det_held, np.array([0, 5], dtype=np.int32))
    E1, _ = dets[1].read()
    assert parity_err(E1[[0, 5]], Eh) <= 1e-4
    for dd in dets:
        dd.close()
    ref.close()
    del keep


def test_linear_interpolation_chunks_and_particle_splits():
    """Step chunks of 64 and 100 intervals and two calls over particle halves: each chunk starts
    from the field of the sample before it, so the result does not depend on the split."""
    import torch
    tr, det = _linear_cases()[0]
    full = rd.RadiationDetector.from_workload(det, "mixed")
    full.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
                 tr.t0, tr.dt)
    Ef, Bf = full.read()
    full.close()
    for chunk in (64, 100):
        d = rd.RadiationDetector.from_workload(det, "mixed")
        d.set_chunk(chunk)
        for sl in (slice(0, 2), slice(2, tr.n_part)):
            one = tr.subset(range(tr.n_part)[sl])
            d.deposit(torch.from_numpy(one.x).cuda(), torch.from_numpy(one.u).cuda(),
                      torch.from_numpy(one.q).cuda(), one.t0, one.dt)
        E, B = d.read()
        d.close()
        assert parity_err(E, Ef) <= 2e-6 and parity_err(B, Bf) <= 2e-6


# --------------------------------------------------------------------------------------------
# quadratic-in-time interpolation (RD_QUADRATIC)
# --------------------------------------------------------------------------------------------
def _quadratic_cases():
    out = []
    for tr, det in _linear_cases():
        det.flags = (det.flags & ~W.RD_LINEAR) | W.RD_QUADRATIC
        out.append((tr, det))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [0, 1, 2, 3])
def test_quadratic_interpolation(precision, case):
    """RD_QUADRATIC (the quadratic through the fields of samples k-2, k-1, k) on the four cases of the
    linear interpolation -- window cuts and per-cell origins, the undulator ensemble, intervals
    spanning several bins in tracked and untracked blocks, the far-field limit: every cell against the
    oracle (clipped counts exact in FP64)."""
    tr, det = _quadratic_cases()[case]
    check(tr, det, precision)


def test_quadratic_chunks_streams_and_batch():
    """RD_QUADRATIC does not depend on how the work is split: step chunks of 64 and 100 intervals
    (every chunk starts from the fields of the two samples before it), two calls over particle
    halves, the stream in stretches of 1, 1, 7, 64 and the rest (the detector keeps three samples and
    the trajectory's interval count), and one batched launch beside a held problem -- each equals
    the plain call (2e-6), and the plain call the oracle."""
    import torch
    tr, det = _quadratic_cases()[0]
    xd, ud, qd = (torch.from_numpy(a).cuda() for a in (tr.x, tr.u, tr.q))
    ref = rd.RadiationDetector.from_workload(det, "mixed")
    ref.deposit(xd, ud, qd, tr.t0, tr.dt)
    Er, Br = ref.read()
    Eo, Bo, _ = oracle.deposit(tr, det)
    assert parity_err(Er, Eo) <= TOL["mixed"] and parity_err(Br, Bo) <= TOL["mixed"]
    for chunk in (64, 100):
        d = rd.RadiationDetector.from_workload(det, "mixed")
        d.set_chunk(chunk)
        for sl in (slice(0, 2), slice(2, tr.n_part)):
            one = tr.subset(range(tr.n_part)[sl])
            d.deposit(torch.from_numpy(one.x).cuda(), torch.from_numpy(one.u).cuda(),
                      torch.from_numpy(one.q).cuda(), one.t0, one.dt)
        E, B = d.read()
        d.close()
        assert parity_err(E, Er) <= 2e-6 and parity_err(B, Br) <= 2e-6, chunk
    for precision in ("mixed", "fp64"):
        d = rd.RadiationDetector.from_workload(det, precision)
        k = 0
        for m in (1, 1, 7, 64, tr.n_samples):
            b = min(tr.n_samples, k + m)
            d.deposit_stream(xd[:, k:b].contiguous(), ud[:, k:b].contiguous(), qd, tr.t0 + k * tr.dt, tr.dt)
            k = b
            if k >= tr.n_samples:
                break
        E, B = d.read()
        d.close()
        tol = 2e-6 if precision == "mixed" else 1e-10
        want = (Er, Br) if precision == "mixed" else (Eo, Bo)
        assert parity_err(E, want[0]) <= tol and parity_err(B, want[1]) <= tol, precision
    det_held = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins, W.RD_NEAR | W.RD_FAR)
    dets = [rd.RadiationDetector.from_workload(det, "mixed"), rd.RadiationDetector.from_workload(det_held, "mixed")]
    keep = rd.deposit_batch(dets, [(xd, ud, qd, tr.t0, tr.dt)] * 2)
    E0, B0 = dets[0].read()
    assert parity_err(E0, Er) <= 2e-6 and parity_err(B0, Br) <= 2e-6
    for dd in dets:
        dd.close()
    ref.close()
    del keep


def test_measure_fma_peaks_plausible():
    """The FMA microbenchmark (roofline denominator): FP32 within the 152-SM part's range
    (at most 152 x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s; a run far below that would be a
    broken probe), FP64 positive and well below FP32 on this part."""
    f32, f64 = rd.rd_measure_fma_peaks()
    assert 20.0 < f32 < 85.0, f32
    assert 0.05 < f64 < f32, (f32, f64)


def test_bounded_wait_runs_out_and_reports():
    """The kernels' bounded mbarrier wait, on a phase that nothing completes, gives up after its limit
    and the expiry comes back as RD_ERR_TIMEOUT; the context stays usable (a deposit afterwards
    matches the oracle)."""
    import time
    t = time.perf_counter()
    assert rd.rd_check_bounded_wait(20) == rd.RD_ERR_TIMEOUT
    assert time.perf_counter() - t < 5.0
    assert "bounded wait" in rd.rd_last_error()
    tr = W.random_smooth(2, 60, 0.03, seed=31)
    det = W.Detector(W.spherical_cap(3, 12.0, 0.5), None, 9.0, 0.02, 300)
    check(tr, det, "mixed")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_plasma_mirror_full_plane_and_steps(precision):
    """The plasma-mirror configuration with its full detector (256x256 plane x 4096 bins of 5 dt,
    per-cell time origins) and its full 10^4 steps, for the first 10^3 of its 10^5 electrons
    (generated on the device by the generator a CPU test pins to the host one); 8 cells against the
    FP64 oracle.  The mixed path deposits the whole plane (6.6e11 deposits); the FP64 path runs on a
    detector of the 8 cells only (the whole plane in FP64 takes minutes)."""
    import torch
    n_steps = 10_000
    x, u, q, (t0, dt) = W.plasma_mirror_surface_torch(slice(0, 1000), n_part=100_000, n_steps=n_steps)
    det = W.plasma_mirror_detector(dt)
    rng = np.random.default_rng(31)
    sel = np.sort(rng.choice(det.n_pix, 8, replace=False)).astype(np.int32)
    if precision == "mixed":
        d = rd.RadiationDetector.from_workload(det, "mixed")
        d.deposit(x, u, q, t0, dt)
        E, B = d.read("float32", "cuda")
        idx = torch.from_numpy(sel.astype(np.int64)).cuda()
        E, B = E[idx].double().cpu().numpy(), B[idx].double().cpu().numpy()
    else:
        d = rd.RadiationDetector.from_workload(det.subset(sel), "fp64")
        d.deposit(x, u, q, t0, dt)
        E, B = d.read()
    st = d.stats()
    d.close()
    assert st.device_errors == 0
    tr = W.Trajectories(x.cpu().numpy(), u.cpu().numpy(), q.cpu().numpy(), t0, dt)
    del x, u
    Eo, Bo, _ = oracle.deposit(tr, det, sel)
    assert np.abs(Eo).max() > 0
    assert parity_err(E, Eo) <= TOL[precision] and parity_err(B, Bo) <= TOL[precision]
