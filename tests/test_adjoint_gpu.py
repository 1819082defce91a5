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
TOL_COMP = 1e-6          # the compensated adjoint: the gradient bar of the adjoint workload
TOL_ADJ = {"mixed": TOL, "comp": TOL_COMP, "fp64": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rd.load_library()
    oracle.build()


def gpu_adjoint(tr, det, gE, gB, precision="mixed"):
    """precision: "mixed" (FP32 adjoint), "comp" (RD_MIXED detector, RD_ADJ_COMPENSATED) or "fp64"."""
    import torch
    d = rd.RadiationDetector.from_workload(det, "mixed" if precision == "comp" else precision)
    if precision == "comp":
        d.set_adjoint_mode("compensated")
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


@pytest.mark.parametrize("precision", ["mixed", "comp", "fp64"])
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


@pytest.mark.parametrize("precision", ["mixed", "comp", "fp64"])
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


@pytest.mark.parametrize("precision", ["mixed", "comp", "fp64"])
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


# ---------------------------------------------------------------------------------------------
# compensated adjoint (RD_ADJ_COMPENSATED) on the adjoint workload at full size: the 1e-6 bar
# ---------------------------------------------------------------------------------------------
def _coords(tr, rng, n):
    """n seeded (which, particle, sample, component) coordinates, positions and momenta alternating."""
    out = []
    for i in range(n):
        out.append((("x", "u")[i % 2], int(rng.integers(0, tr.n_part)), int(rng.integers(0, tr.n_samples)),
                    int(rng.integers(0, 3))))
    return out


@pytest.fixture(scope="module")
def adjoint_full():
    """The adjoint workload (1e4 undulator electrons x 2000 steps, 64x64 x 1024) with a seeded
    smooth seed standing in for the misfit E - E_target, its compensated and FP32 gradients."""
    rng = np.random.default_rng(55)
    tr, det = _adjoint_config()
    gE = _smooth_seed(det, rng)
    gxc, guc = gpu_adjoint(tr, det, gE, None, "comp")
    gxm, gum = gpu_adjoint(tr, det, gE, None, "mixed")
    return tr, det, gE, (gxc, guc), (gxm, gum)


def test_compensated_adjoint_full_size_50_coordinates(adjoint_full):
    """The compensated adjoint at full size against the oracle's exact (complex-step) derivative
    at 50 seeded coordinates (25 positions, 25 momenta, any sample including the first and the
    chunk boundaries): relative L2 <= 1e-6 for positions and for momenta separately, every
    coordinate within 2e-5 of its own size or of the RMS."""
    tr, det, gE, (gxc, guc), (gxm, gum) = adjoint_full
    rng = np.random.default_rng(505)
    coords = _coords(tr, rng, 46) + [("x", 17, 250, 2), ("u", 17, 250, 1), ("x", 33, 0, 0), ("u", 9, 2000, 2)]
    want = oracle_vjp(tr, det, gE, None, coords)
    got = np.array([(gxc if w == "x" else guc)[p, k, c] for (w, p, k, c) in coords])
    fp32 = np.array([(gxm if w == "x" else gum)[p, k, c] for (w, p, k, c) in coords])
    isx = np.array([w == "x" for (w, _, _, _) in coords])
    ex, eu = parity_err(got[isx], want[isx]), parity_err(got[~isx], want[~isx])
    print(f"compensated: x {ex:.3e}  u {eu:.3e};  FP32 adjoint: x {parity_err(fp32[isx], want[isx]):.3e}  "
          f"u {parity_err(fp32[~isx], want[~isx]):.3e}")
    assert ex <= TOL_COMP and eu <= TOL_COMP, (ex, eu)


def test_compensated_adjoint_momenta_against_oracle_differences(adjoint_full):
    """Fourth-order central differences of L = sum_b gE . E_b through the FP64 oracle's deposit of the
    perturbed electron alone (the exact difference of its contribution; the others do not depend on
    the coordinate) at 25 seeded momentum coordinates.  A momentum moves no arrival time (those
    depend on positions only), so the deposit is smooth in it and the quotient needs no bin-edge
    exclusion.  Bar 1e-6 relative L2."""
    tr, det, gE, (gxc, guc), _ = adjoint_full
    rng = np.random.default_rng(606)
    errs, refs = [], []
    for _ in range(25):
        p, k, c = int(rng.integers(0, tr.n_part)), int(rng.integers(1, tr.n_samples)), int(rng.integers(0, 3))
        one = tr.subset([p])
        h = 1e-5 * max(1.0, abs(one.u[0, k, c]))
        vals = {}
        for m in (-2, -1, 1, 2):
            pert = W.Trajectories(one.x, one.u.copy(), one.q, one.t0, one.dt)
            pert.u[0, k, c] = one.u[0, k, c] + m * h
            E, _, _ = oracle.deposit(pert, det)
            vals[m] = float(np.sum(E * gE))
        fd = (8.0 * (vals[1] - vals[-1]) - (vals[2] - vals[-2])) / (12.0 * h)
        errs.append(guc[p, k, c] - fd)
        refs.append(fd)
    assert np.linalg.norm(errs) <= TOL_COMP * np.linalg.norm(refs), (errs, refs)


def test_compensated_adjoint_positions_against_oracle_differences():
    """Central differences through the long double oracle (the exact difference of the perturbed
    electron's contribution) at 12 seeded position coordinates of the full-size adjoint workload.
    A position moves its sample's arrival time, and the deposit has a kink where that arrival
    crosses a bin edge, so the seed lives on 64 cells and each coordinate's step is a quarter of
    its arrival's distance to the nearest bin edge on those cells (the long double evaluation keeps
    the quotient's rounding far below the bar at that step).  Bar 1e-6 relative L2."""
    import math as _m
    rng = np.random.default_rng(707)
    tr, det = _adjoint_config()
    sel = np.sort(rng.choice(det.n_pix, 64, replace=False)).astype(np.int32)
    g_full = np.zeros((det.n_pix, det.n_bins, 3))
    g_full[sel] = rng.normal(size=(64, det.n_bins, 3))
    gx, _ = gpu_adjoint(tr, det, g_full, None, "comp")
    g = g_full[sel]
    inv = 1.0 / det.dt_det
    errs, refs = [], []
    tries = 0
    while len(refs) < 12 and tries < 100:
        tries += 1
        p, k, c = int(rng.integers(0, tr.n_part)), int(rng.integers(0, tr.n_samples)), int(rng.integers(0, 3))
        # distance (bins) from sample k's arrival to the nearest bin edge, over the seeded cells
        dist = min(0.5 - abs(v - _m.floor(v) - 0.5) for v in
                   (oracle.bin_coord(tr.t0, k, tr.dt, tr.x[p, k], det.pix_pos[j],
                                     det.t_min + (0.0 if det.pix_t0 is None else det.pix_t0[j]), inv) for j in sel))
        h = 0.25 * dist * det.dt_det                       # |d t' / d x| <= 1
        if h < 1e-9:
            continue
        one = tr.subset([p])
        vals = []
        for sgn in (1.0, -1.0):
            pert = W.Trajectories(one.x.copy(), one.u, one.q, one.t0, one.dt)
            pert.x[0, k, c] = one.x[0, k, c] + sgn * h
            E, _, _ = oracle.deposit_ext(pert, det, sel)
            vals.append((float(np.sum(E * g)), pert.x[0, k, c]))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        errs.append(gx[p, k, c] - fd)
        refs.append(fd)
    assert len(refs) == 12
    assert np.linalg.norm(errs) <= TOL_COMP * np.linalg.norm(refs), (errs, refs)


def test_compensated_adjoint_against_fp64_adjoint_every_coordinate():
    """20 electrons of the adjoint workload, every coordinate: the compensated adjoint against the
    plain FP64 adjoint (relative L2 <= 1e-6 and every coordinate within 2e-5 of its size or the RMS;
    the FP32 adjoint's error on the same set is printed)."""
    rng = np.random.default_rng(21)
    tr, det = _adjoint_config(n_part=20)
    gE = rng.normal(size=(det.n_pix, det.n_bins, 3))
    gxc, guc = gpu_adjoint(tr, det, gE, None, "comp")
    gxm, gum = gpu_adjoint(tr, det, gE, None, "mixed")
    gx64, gu64 = gpu_adjoint(tr, det, gE, None, "fp64")
    print(f"compensated vs FP64 adjoint: x {parity_err(gxc, gx64):.3e} u {parity_err(guc, gu64):.3e}; "
          f"FP32: x {parity_err(gxm, gx64):.3e} u {parity_err(gum, gu64):.3e}")
    assert parity_err(gxc, gx64) <= TOL_COMP and parity_err(guc, gu64) <= TOL_COMP


def test_adjoint_mode_arguments():
    tr = W.random_smooth(1, 10, 0.02, seed=1)
    det = W.Detector(W.spherical_cap(2, 10.0, 0.3), None, 8.0, 0.02, 100)
    d = rd.RadiationDetector.from_workload(det, "fp64")
    with pytest.raises(rd.RDError) as ei:
        d.set_adjoint_mode("compensated")
    assert ei.value.status == rd.RD_ERR_STATE
    d.close()
    d = rd.RadiationDetector.from_workload(det, "mixed")
    with pytest.raises(rd.RDError) as ei:
        rd.rd_set_adjoint_mode(d.handle, 7)
    assert ei.value.status == rd.RD_ERR_ARG
    d.set_adjoint_mode("compensated")
    d.set_adjoint_mode("fp32")
    d.close()
