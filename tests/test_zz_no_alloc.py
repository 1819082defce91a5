"""Allocation-free deposit (rd_deposit_noalloc) through the C ABI.

This entry point is for callers that cannot call cudaMalloc: a particle-in-cell code whose device
memory is a pool reserved at start-up, a host framework whose allocator owns the device, or a loop
that must not pay the synchronisation cudaMalloc / cudaFree can cause.  Its output must equal the
detector path's (rd_deposit_trajectories on an RD_MIXED detector) within the 2e-6 relative L2 that
the same-arithmetic comparisons of this suite use (only the order of FP32 reductions differs), on
two calls in a row: the second call reuses the library's scratch array as the first left it.
"""
import numpy as np
import pytest

import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rd.load_library()


def _cases():
    tr1, det1 = W.config_undulator(n_part=6, n_steps=1500, n_side=24, n_bins=512, seed=3)
    rng = np.random.default_rng(4)
    tr2 = W.random_smooth(5, 700, 0.02, max_u=2.5, seed=4)
    pos = rng.normal(size=(333, 3)) * 20.0
    det2 = W.Detector(pos, rng.uniform(-1.0, 1.0, 333), 10.0, 0.02, 600)   # cuts some arrivals
    return [(tr1, det1), (tr2, det2)]


@pytest.mark.parametrize("case", [0, 1])
def test_noalloc_matches_detector_path_on_two_calls(case):
    import torch
    tr, det = _cases()[case]
    x, u, q = (torch.from_numpy(a).cuda() for a in (tr.x, tr.u, tr.q))
    ref = rd.RadiationDetector.from_workload(det, "mixed")
    ref.deposit(x, u, q, tr.t0, tr.dt)
    Er, Br = ref.read()
    traj, keep = ref.traj_struct(x, u, q, tr.t0, tr.dt)
    pos = torch.from_numpy(det.pix_pos).cuda()
    t0 = None if det.pix_t0 is None else torch.from_numpy(det.pix_t0).cuda()
    for _ in range(2):
        fields = torch.zeros((det.n_pix, det.n_bins, 8), dtype=torch.float32, device="cuda")
        err = rd.rd_deposit_noalloc(pos.data_ptr(), None if t0 is None else t0.data_ptr(), det.n_pix,
                                    det.t_min, det.dt_det, det.n_bins, det.flags, traj, fields.data_ptr())
        assert err == 0
        f = fields.double().cpu().numpy()
        assert parity_err(f[..., 0:3], Er) <= TOL
        assert parity_err(f[..., 3:6], Br) <= TOL
        assert np.all(f[..., 6:] == 0)
    ref.close()
    del keep


def test_noalloc_limits_and_input_errors():
    import torch
    tr = W.random_smooth(1, 20, 0.05, seed=1)
    x, u = torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda()
    det = W.Detector(np.array([[10.0, 0.0, 0.0]]), None, 0.0, 0.1, 100)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    traj, keep = d.traj_struct(x, u, None, tr.t0, tr.dt)
    fields = torch.zeros((1, 100, 8), dtype=torch.float32, device="cuda")
    pos = torch.from_numpy(det.pix_pos).cuda()
    # more cells than the scratch holds: rejected before any work
    with pytest.raises(rd.RDError) as ei:
        rd.rd_deposit_noalloc(pos.data_ptr(), None, 262145, 0.0, 0.1, 100, 3, traj, fields.data_ptr())
    assert ei.value.status == rd.RD_ERR_ARG and "262144" in str(ei.value)
    # a superluminal chord is reported through the error bits of this call only
    bad = tr.x.copy()
    bad[0, 7] = bad[0, 6] + np.array([0.06, 0.0, 0.0])
    tb, kb = d.traj_struct(torch.from_numpy(bad).cuda(), u, None, tr.t0, tr.dt)
    err = rd.rd_deposit_noalloc(pos.data_ptr(), None, 1, 0.0, 0.1, 100, 3, tb, fields.data_ptr())
    assert err & (1 << rd.RD_ERR_INPUT)
    err = rd.rd_deposit_noalloc(pos.data_ptr(), None, 1, 0.0, 0.1, 100, 3, traj, fields.data_ptr())
    assert err == 0
    d.close()
    del keep, kb


def _sampled_oracle(tr, det, f, n_cells, seed):
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(det.n_pix, size=min(n_cells, det.n_pix), replace=False)).astype(np.int32)
    Eo, Bo, _ = oracle.deposit(tr, det, sel)
    return parity_err(f[sel, :, 0:3], Eo), parity_err(f[sel, :, 3:6], Bo)


@pytest.mark.parametrize("case", [0, 1])
def test_noalloc_against_oracle_sampled_cells(case):
    """The allocation-free deposit against the FP64 oracle on 8 random cells: the mixed path's bar
    (1e-4 relative L2, every element within 2e-3 of the oracle's RMS)."""
    import torch
    tr, det = _cases()[case]
    x, u, q = (torch.from_numpy(a).cuda() for a in (tr.x, tr.u, tr.q))
    d = rd.RadiationDetector.from_workload(det, "mixed")
    traj, keep = d.traj_struct(x, u, q, tr.t0, tr.dt)
    pos = torch.from_numpy(det.pix_pos).cuda()
    t0 = None if det.pix_t0 is None else torch.from_numpy(det.pix_t0).cuda()
    fields = torch.zeros((det.n_pix, det.n_bins, 8), dtype=torch.float32, device="cuda")
    err = rd.rd_deposit_noalloc(pos.data_ptr(), None if t0 is None else t0.data_ptr(), det.n_pix, det.t_min,
                                det.dt_det, det.n_bins, det.flags, traj, fields.data_ptr())
    assert err == 0
    eE, eB = _sampled_oracle(tr, det, fields.double().cpu().numpy(), 8, 10 + case)
    assert eE <= 1e-4 and eB <= 1e-4, (eE, eB)
    d.close()
    del keep


def test_noalloc_several_particle_passes():
    """64 electrons x 20000 intervals: their records (64 x 20001 x 64 B = 81.9 MB) exceed the 56 MiB
    record area of the scratch array, so one call runs two precompute + deposit passes (45 and 19
    electrons) through the same scratch on one stream.  Against the detector path on every cell, on
    two calls in a row, and against the FP64 oracle on 6 cells."""
    import torch
    tr, det = W.config_undulator(n_part=64, n_steps=20000, n_side=5, n_bins=1024, seed=6)
    assert tr.n_part * tr.n_samples * 64 > 56 * 2**20
    x, u, q = (torch.from_numpy(a).cuda() for a in (tr.x, tr.u, tr.q))
    ref = rd.RadiationDetector.from_workload(det, "mixed")
    ref.deposit(x, u, q, tr.t0, tr.dt)
    Er, Br = ref.read()
    traj, keep = ref.traj_struct(x, u, q, tr.t0, tr.dt)
    pos = torch.from_numpy(det.pix_pos).cuda()
    for _ in range(2):
        fields = torch.zeros((det.n_pix, det.n_bins, 8), dtype=torch.float32, device="cuda")
        err = rd.rd_deposit_noalloc(pos.data_ptr(), None, det.n_pix, det.t_min, det.dt_det, det.n_bins, det.flags,
                                    traj, fields.data_ptr())
        assert err == 0
        f = fields.double().cpu().numpy()
        assert parity_err(f[..., 0:3], Er) <= TOL
        assert parity_err(f[..., 3:6], Br) <= TOL
    eE, eB = _sampled_oracle(tr, det, f, 6, 12)
    assert eE <= 1e-4 and eB <= 1e-4, (eE, eB)
    ref.close()
    del keep


def test_noalloc_non_finite_cell_is_reported():
    """A cell with a non-finite position is reported through the call's error bits (the detector
    path refuses such a cell when the detector is created)."""
    import torch
    tr = W.random_smooth(1, 20, 0.05, seed=1)
    x, u = torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda()
    det = W.Detector(np.array([[10.0, 0.0, 0.0], [0.0, 10.0, 0.0]]), None, 0.0, 0.1, 100)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    traj, keep = d.traj_struct(x, u, None, tr.t0, tr.dt)
    fields = torch.zeros((2, 100, 8), dtype=torch.float32, device="cuda")
    bad = det.pix_pos.copy()
    bad[1, 2] = np.nan
    pos = torch.from_numpy(bad).cuda()
    err = rd.rd_deposit_noalloc(pos.data_ptr(), None, 2, 0.0, 0.1, 100, 3, traj, fields.data_ptr())
    assert err & (1 << rd.RD_ERR_INPUT)
    pos = torch.from_numpy(det.pix_pos).cuda()
    err = rd.rd_deposit_noalloc(pos.data_ptr(), None, 2, 0.0, 0.1, 100, 3, traj, fields.data_ptr())
    assert err == 0
    d.close()
    del keep
