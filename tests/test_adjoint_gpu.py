"""Adjoint (gather) kernel through the C ABI against the oracle's exact derivative.

The oracle's complex-step derivative d E_det / d theta of one particle's contribution, projected
on the same seed (dE . gE + dB . gB), is the exact directional derivative of the FP64 deposit.
The GPU adjoint differentiates the mixed-precision deposit (FP32 field arithmetic).  Its error is
set by FP32 rounding amplified in the transposed backward difference: the gradient at sample k
holds differences of neighbouring-sample terms, (dF/dbetadot_k - dF/dbetadot_{k+1})/dt and
(F_k - F_{k+1}).g, each rounded separately, so a per-step relative error of ~1e-7 grows by the
ratio of those terms to their difference (measured: ~3e-6 for d/dx, ~1.3e-5 for d/du).  The bar
is a relative L2 error of 5e-5 over the compared coordinates.  The FP64 adjoint (an RD_FP64
detector) differentiates the plain FP64 deposit with the same algebra in FP64: bar 1e-9.  Seeds
are seeded synthetic arrays (never taken from the GPU).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err

pytestmark = pytest.mark.gpu

TOL = 5e-5
TOL_ADJ = {"mixed": TOL, "fp64": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rd.load_library()
    oracle.build()


def gpu_adjoint(tr, det, gE, gB, precision="mixed"):
    import torch
    d = rd.RadiationDetector.from_workload(det, precision)
    x = torch.from_numpy(tr.x).cuda()
    u = torch.from_numpy(tr.u).cuda()
    q = torch.from_numpy(tr.q).cuda()
    gx, gu = d.adjoint(x, u, q, tr.t0, tr.dt, torch.from_numpy(gE).cuda(),
                       None if gB is None else torch.from_numpy(gB).cuda())
    d.synchronize()
    d.close()
    return gx.cpu().numpy(), gu.cpu().numpy()


def oracle_vjp(tr, det, gE, gB, coords, sel=None, threads=None):
    out = []
    for (which, p, k, c) in coords:
        dE, dB = oracle.deposit_dir(tr, det, p, k, which, c, sel=sel, n_threads=threads)
        v = float(np.sum(dE * gE))
        if gB is not None:
            v += float(np.sum(dB * gB))
        out.append(v)
    return np.array(out)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("seed", [1, 2])
def test_adjoint_all_coordinates_small(seed, precision):
    """Every x and u coordinate of 2 particles x 150 intervals, 9 cells, window with margins."""
    rng = np.random.default_rng(seed)
    tr = W.random_smooth(2, 150, 0.02, max_u=2.5, seed=seed)
    det = W.Detector(W.spherical_cap(3, 20.0, 0.5), None, 16.0, 0.011, 900)
    gE = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gB = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gx, gu = gpu_adjoint(tr, det, gE, gB, precision)
    coords_x = [("x", p, k, c) for p in range(tr.n_part) for k in range(tr.n_samples) for c in range(3)]
    coords_u = [("u", p, k, c) for p in range(tr.n_part) for k in range(tr.n_samples) for c in range(3)]
    ox = oracle_vjp(tr, det, gE, gB, coords_x, threads=4)
    ou = oracle_vjp(tr, det, gE, gB, coords_u, threads=4)
    ex, eu = parity_err(gx.reshape(-1), ox), parity_err(gu.reshape(-1), ou)
    assert ex <= TOL_ADJ[precision] and eu <= TOL_ADJ[precision], (ex, eu)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_adjoint_clipped_window_and_cell_origins(precision):
    """Window that cuts arrivals at both ends, per-cell time origins, E-only seed."""
    rng = np.random.default_rng(7)
    tr = W.random_smooth(2, 120, 0.02, max_u=2.0, seed=7)
    pos = W.spherical_cap(3, 15.0, 0.6)
    t0 = rng.uniform(-0.3, 0.3, pos.shape[0])
    det = W.Detector(pos, t0, 15.8, 0.009, 150)
    gE = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gx, gu = gpu_adjoint(tr, det, gE, None, precision)
    coords_x = [("x", p, k, c) for p in range(tr.n_part) for k in range(tr.n_samples) for c in range(3)]
    coords_u = [("u", p, k, c) for p in range(tr.n_part) for k in range(tr.n_samples) for c in range(3)]
    ox = oracle_vjp(tr, det, gE, None, coords_x, threads=4)
    ou = oracle_vjp(tr, det, gE, None, coords_u, threads=4)
    tol = TOL_ADJ[precision]
    assert parity_err(gx.reshape(-1), ox) <= tol and parity_err(gu.reshape(-1), ou) <= tol


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_adjoint_cells_missing_the_window(precision):
    """130 cells (two cell blocks, the second ragged); every third cell's time axis lies far after
    all its arrivals.  Those cells contribute exactly nothing (a seed on them alone gives exact
    zeros), and the gradient of the mixed set matches the oracle."""
    rng = np.random.default_rng(11)
    tr = W.random_smooth(2, 140, 0.02, max_u=2.0, seed=11)
    pos = rng.normal(size=(130, 3)) * 4.0 + np.array([0.0, 0.0, 14.0])
    t0 = rng.uniform(-0.2, 0.2, 130)
    dead = np.arange(130) % 3 == 0
    t0[dead] += 60.0
    det = W.Detector(pos, t0, 13.0, 0.01, 400)
    g = rng.normal(size=(det.n_pix, det.n_bins, 3))
    g_dead = np.where(dead[:, None, None], g, 0.0)
    gx, gu = gpu_adjoint(tr, det, g_dead, g_dead, precision)
    assert not np.any(gx) and not np.any(gu)
    gx, gu = gpu_adjoint(tr, det, g, None, precision)
    pick = rng.choice(tr.n_part * tr.n_samples * 3, size=60, replace=False)
    coords = [(w, int(i // (tr.n_samples * 3)), int(i // 3 % tr.n_samples), int(i % 3)) for i in pick
              for w in ("x", "u")]
    ref = oracle_vjp(tr, det, g, None, coords, threads=4)
    got = np.array([(gx if w == "x" else gu)[p, k, c] for (w, p, k, c) in coords])
    assert np.any(ref != 0.0)
    assert parity_err(got, ref) <= TOL_ADJ[precision]


def _adjoint_config(n_part=10_000):
    """Undulator electrons (gamma 10, K 1) x 2000 steps, 64x64 cap x 1024 bins."""
    return W.config_undulator(n_part=n_part, n_steps=2000, n_side=64, n_bins=1024, gamma=10.0, K=1.0,
                              n_periods=10.0, distance=1e4, seed=5)


def _smooth_seed(det, rng):
    b = np.arange(det.n_bins)[None, :, None]
    j = np.arange(det.n_pix)[:, None, None]
    c = np.arange(3)[None, None, :]
    return (np.sin(2 * math.pi * b / 41.0 + 0.37 * j + 1.3 * c) +
            0.3 * rng.normal(size=(det.n_pix, det.n_bins, 3)))


def test_adjoint_full_size_sampled_coordinates():
    """The adjoint workload at full size (1e4 electrons x 2000 steps x 64x64 x 1024) through the
    C ABI; the oracle's exact derivative at 16 random (particle, sample, component) coordinates."""
    rng = np.random.default_rng(5)
    tr, det = _adjoint_config()
    gE = _smooth_seed(det, rng)
    gx, gu = gpu_adjoint(tr, det, gE, None)
    coords = []
    for _ in range(16):
        p = int(rng.integers(0, tr.n_part))
        k = int(rng.integers(1, tr.n_samples - 1))
        coords.append((["x", "u"][len(coords) % 2], p, k, int(rng.integers(0, 3))))
    want = oracle_vjp(tr, det, gE, None, coords)
    got = np.array([(gx if w == "x" else gu)[p, k, c] for (w, p, k, c) in coords])
    assert parity_err(got, want) <= TOL, (got, want)


def _crosses_bin_edge(tr, det, p, k, c, h):
    """True if moving x[p][k][c] by +-h moves the arrival time of sample k at some cell across a
    bin edge (there the deposit is only piecewise smooth and a difference quotient is wrong)."""
    inv = 1.0 / det.dt_det
    for sgn in (1.0, -1.0):
        xs = tr.x[p, k].copy()
        xs[c] += sgn * h
        for j in range(det.n_pix):
            T0 = det.t_min + (0.0 if det.pix_t0 is None else det.pix_t0[j])
            a = oracle.bin_coord(tr.t0, k, tr.dt, tr.x[p, k], det.pix_pos[j], T0, inv)
            b = oracle.bin_coord(tr.t0, k, tr.dt, xs, det.pix_pos[j], T0, inv)
            if math.floor(a) != math.floor(b):
                return True
    return False


def test_mixed_adjoint_against_fp64_adjoint_every_coordinate():
    """20 electrons of the adjoint workload (R = 1e4, 64x64 cells x 1024 bins), every coordinate:
    the mixed adjoint against the FP64 adjoint.  The derivative through an arrival time takes the
    seed of the arrival's bin, so an arrival the FP32 walk put on the wrong side of a bin edge
    would show as an outlier of order one; the mixed kernel takes such bins from Eq. 2 in FP64.
    Bars: relative L2 5e-5 and no coordinate off by more than 1e-3 of the RMS."""
    rng = np.random.default_rng(21)
    tr, det = _adjoint_config(n_part=20)
    gE = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gxm, gum = gpu_adjoint(tr, det, gE, None, "mixed")
    gx64, gu64 = gpu_adjoint(tr, det, gE, None, "fp64")
    for a, b in ((gxm, gx64), (gum, gu64)):
        assert parity_err(a.reshape(-1), b.reshape(-1)) <= 5e-5
        assert np.max(np.abs(a - b)) <= 1e-3 * np.sqrt(np.mean(b * b))


def test_adjoint_against_fp64_central_differences():
    """Central differences of sum_b g_b . E_b through the FP64 GPU deposit of the perturbed particle
    alone (the other particles do not depend on the coordinate), at coordinates whose perturbation
    keeps every arrival time inside its bin.  Bar 2e-4: the FP32 adjoint's rounding (module
    docstring) plus the difference quotient's error (at R = 1e4 a position step of 1e-8 changes R
    by ~1e-8 against R's own FP64 rounding of ~1e-12, so the quotient itself is good to ~1e-4)."""
    import torch
    rng = np.random.default_rng(11)
    tr, det = _adjoint_config(n_part=64)
    gE = _smooth_seed(det, rng)
    gx, gu = gpu_adjoint(tr, det, gE, None)
    f64 = rd.RadiationDetector.from_workload(det, "fp64")
    errs, refs = [], []
    tried = 0
    while len(refs) < 12 and tried < 60:
        tried += 1
        p = int(rng.integers(0, tr.n_part))
        k = int(rng.integers(2, tr.n_samples - 2))
        c = int(rng.integers(0, 3))
        which = "x" if tried % 2 == 0 else "u"
        arr = tr.x if which == "x" else tr.u
        h = (1e-8 if which == "x" else 1e-6) * max(1.0, abs(arr[p, k, c]))
        if which == "x" and _crosses_bin_edge(tr, det, p, k, c, h):
            continue
        one = tr.subset([p])
        vals = []
        for sgn in (1.0, -1.0):
            pert = W.Trajectories(one.x.copy(), one.u.copy(), one.q, one.t0, one.dt)
            (pert.x if which == "x" else pert.u)[0, k, c] += sgn * h
            f64.zero()
            f64.deposit(torch.from_numpy(pert.x).cuda(), torch.from_numpy(pert.u).cuda(),
                        torch.from_numpy(pert.q).cuda(), pert.t0, pert.dt)
            E, _ = f64.read("float64", "cpu")
            vals.append(float(np.sum(E * gE)))
        fd = (vals[0] - vals[1]) / (2 * h)
        g = (gx if which == "x" else gu)[p, k, c]
        errs.append(g - fd)
        refs.append(fd)
    f64.close()
    assert len(refs) >= 8
    assert np.linalg.norm(errs) <= 2e-4 * np.linalg.norm(refs), (errs, refs)


def test_fp64_adjoint_against_central_differences():
    """The FP64 adjoint against fourth-order central differences (error O(h^4)) of
    sum_b (g_E . E_b + g_B . B_b) through the FP64 GPU deposit of the perturbed particle, on a
    detector at R ~ 15 where the quotient is well conditioned; coordinates whose perturbations move
    an arrival time across a bin edge are skipped.  Bar 1e-6 relative L2."""
    import torch
    rng = np.random.default_rng(12)
    tr = W.random_smooth(3, 200, 0.02, max_u=2.0, seed=12)
    det = W.Detector(W.spherical_cap(3, 15.0, 0.5), None, 11.0, 0.01, 1200)
    gE = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gB = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gx, gu = gpu_adjoint(tr, det, gE, gB, "fp64")
    f64 = rd.RadiationDetector.from_workload(det, "fp64")

    def loss(one):
        f64.zero()
        f64.deposit(torch.from_numpy(one.x).cuda(), torch.from_numpy(one.u).cuda(),
                    torch.from_numpy(one.q).cuda(), one.t0, one.dt)
        E, B = f64.read("float64", "cpu")
        return float(np.sum(E * gE) + np.sum(B * gB))

    errs, refs = [], []
    tried = 0
    while len(refs) < 16 and tried < 80:
        tried += 1
        p = int(rng.integers(0, tr.n_part))
        k = int(rng.integers(2, tr.n_samples - 2))
        c = int(rng.integers(0, 3))
        which = "x" if tried % 2 == 0 else "u"
        h = 1e-5
        if which == "x" and _crosses_bin_edge(tr, det, p, k, c, 2 * h):
            continue
        one = tr.subset([p])
        vals = {}
        for m in (-2, -1, 1, 2):
            pert = W.Trajectories(one.x.copy(), one.u.copy(), one.q, one.t0, one.dt)
            (pert.x if which == "x" else pert.u)[0, k, c] += m * h
            vals[m] = loss(pert)
        fd = (8.0 * (vals[1] - vals[-1]) - (vals[2] - vals[-2])) / (12.0 * h)
        errs.append((gx if which == "x" else gu)[p, k, c] - fd)
        refs.append(fd)
    f64.close()
    assert len(refs) >= 10
    assert np.linalg.norm(errs) <= 1e-6 * np.linalg.norm(refs), (errs, refs)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autograd_function_matches_adjoint(precision):
    import torch
    tr = W.random_smooth(2, 80, 0.02, max_u=2.0, seed=3)
    det = W.Detector(W.spherical_cap(2, 15.0, 0.5), None, 12.0, 0.012, 600)
    d = rd.RadiationDetector.from_workload(det, precision)
    x = torch.from_numpy(tr.x).cuda().requires_grad_(True)
    u = torch.from_numpy(tr.u).cuda().requires_grad_(True)
    q = torch.from_numpy(tr.q).cuda()
    rng = np.random.default_rng(0)
    wE = torch.from_numpy(rng.normal(size=(det.n_pix, det.n_bins, 3))).cuda()
    E, B = rd.DepositFunction.apply(d, x, u, q, tr.t0, tr.dt)
    loss = (E * wE).sum() + 0.5 * (B * B).sum()
    loss.backward()
    gx, gu = d.adjoint(x.detach(), u.detach(), q, tr.t0, tr.dt, wE, B.detach())
    assert torch.allclose(x.grad, gx, rtol=1e-6, atol=1e-9 * float(gx.abs().max()))
    assert torch.allclose(u.grad, gu, rtol=1e-6, atol=1e-9 * float(gu.abs().max()))
    d.close()


def test_adjoint_rejects_farfield_linear_and_host_inputs():
    import torch
    tr = W.random_smooth(1, 10, 0.02, seed=1)
    for flags in (W.RD_FAR | W.RD_FARFIELD, W.RD_NEAR | W.RD_FAR | W.RD_LINEAR):
        det = W.Detector(W.spherical_cap(2, 10.0, 0.3), None, 8.0, 0.02, 100, flags=flags)
        d = rd.RadiationDetector.from_workload(det, "fp64")
        g = torch.zeros((det.n_pix, det.n_bins, 3), device="cuda")
        with pytest.raises(rd.RDError) as ei:
            d.adjoint(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), None, 0.0, tr.dt, g)
        assert ei.value.status == rd.RD_ERR_STATE
        d.close()
    det = W.Detector(W.spherical_cap(2, 10.0, 0.3), None, 8.0, 0.02, 100)
    d = rd.RadiationDetector.from_workload(det, "fp64")
    g = torch.zeros((det.n_pix, det.n_bins, 3), device="cuda")
    with pytest.raises(ValueError):
        d.adjoint(tr.x, tr.u, None, 0.0, tr.dt, g)
    d.close()
