"""Streamed deposits (rd_deposit_stream): a trajectory handed over in consecutive stretches of
new samples deposits what one call on the whole trajectory deposits.

FP64 detectors evaluate every arrival time and field from its own sample, so stretches change
only the order of the FP64 reductions (bar 1e-12).  RD_MIXED detectors restart their FP32
arrival-time walk from an exact FP64 anchor at the ends of every stretch, which moves values by
rounding only (bar 2e-6, the suite's same-arithmetic bar), and stay within the mixed path's 1e-4
of the oracle.
"""
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


def _case():
    rng = np.random.default_rng(6)
    tr = W.random_smooth(5, 400, 0.02, max_u=2.5, seed=6)
    pos = rng.normal(size=(300, 3)) * 20.0
    pos += 25.0 * pos / np.linalg.norm(pos, axis=1, keepdims=True)
    det = W.Detector(pos, rng.uniform(-1.0, 1.0, 300), 30.0, 0.013, 800)
    return tr, det


def _stretches(n, sizes):
    out, k = [], 0
    for m in sizes:
        if k >= n:
            break
        out.append((k, min(n, k + m)))
        k += m
    if k < n:
        out.append((k, n))
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("linear", [False, True])
def test_stream_equals_single_call(precision, tol, where, linear):
    """Stretches of 1, 1, 7, 64, 1, 150, 3 and the rest; with RD_LINEAR the detector keeps two
    samples per particle so that the first interval of every stretch is interpolated like the
    others."""
    import torch
    tr, det = _case()
    if linear:
        det.flags = W.RD_NEAR | W.RD_FAR | W.RD_LINEAR
    ref = rd.RadiationDetector.from_workload(det, precision)
    ref.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
                tr.t0, tr.dt)
    Er, Br = ref.read()
    ref.close()
    d = rd.RadiationDetector.from_workload(det, precision)
    for a, b in _stretches(tr.n_samples, [1, 1, 7, 64, 1, 150, 3]):
        x, u = np.ascontiguousarray(tr.x[:, a:b]), np.ascontiguousarray(tr.u[:, a:b])
        q = tr.q
        if where == "device":
            x, u, q = torch.from_numpy(x).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(q).cuda()
        d.deposit_stream(x, u, q, tr.t0 + a * tr.dt, tr.dt)
    E, B = d.read()
    assert parity_err(E, Er) <= tol and parity_err(B, Br) <= tol
    if precision == "mixed":
        sel = np.array([0, 77, 150, 299], dtype=np.int32)
        Eo, Bo, _ = oracle.deposit(tr, det, sel)
        assert parity_err(E[sel], Eo) <= 1e-4 and parity_err(B[sel], Bo) <= 1e-4
    d.close()


def test_stream_continuity_checks_and_reset():
    import torch
    tr, det = _case()
    d = rd.RadiationDetector.from_workload(det, "mixed")
    x, u = torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda()
    d.deposit_stream(x[:, :10], u[:, :10], None, tr.t0, tr.dt)
    for bad in (dict(t0=tr.t0 + 12 * tr.dt), dict(dt=1.5 * tr.dt), dict(n_part=3)):
        n = bad.get("n_part", tr.n_part)
        with pytest.raises(rd.RDError) as ei:
            d.deposit_stream(x[:n, 10:20].contiguous(), u[:n, 10:20].contiguous(), None,
                             bad.get("t0", tr.t0 + 10 * tr.dt), bad.get("dt", tr.dt))
        assert ei.value.status == rd.RD_ERR_STATE
    d.deposit_stream(x[:, 10:20].contiguous(), u[:, 10:20].contiguous(), None, tr.t0 + 10 * tr.dt, tr.dt)
    E1, _ = d.read()
    # after a reset the next call starts a new stream: its first sample emits nothing
    d.stream_reset()
    d.zero()
    d.deposit_stream(x[:3, 40:60].contiguous(), u[:3, 40:60].contiguous(), None, tr.t0 + 40 * tr.dt, tr.dt)
    E2, _ = d.read()
    one = rd.RadiationDetector.from_workload(det, "mixed")
    one.deposit(x[:3, 40:60].contiguous(), u[:3, 40:60].contiguous(), None, tr.t0 + 40 * tr.dt, tr.dt)
    E3, _ = one.read()
    assert parity_err(E2, E3) <= 2e-6 and np.abs(E1).max() > 0
    one.close()
    d.close()


def _boris_case():
    rng = np.random.default_rng(17)
    n = 6
    u0 = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(1.0, 3.0, n), rng.uniform(0.5, 2.0, n)], axis=1)
    x0 = rng.normal(size=(n, 3)) * 0.1
    B, qm, dt, n_steps = (0.0, 0.0, 1.5), -1.0, 0.05, 400
    tr = W.boris_uniform_field(x0, u0, n_steps, dt, B, qm)
    pos = rng.normal(size=(300, 3))
    pos = 30.0 * pos / np.linalg.norm(pos, axis=1, keepdims=True)
    t_end = n_steps * dt
    det = W.Detector(pos, None, 30.0 - 25.0, 0.02, int((t_end + 50.0) / 0.02))
    return tr, det, x0, u0, B, qm, dt, n_steps


def test_boris_pusher_matches_the_recurrence():
    """rd_push_boris against the same Boris recurrence in numpy (FP64, 400 steps in chunks of 50):
    samples agree to rounding, |u| is kept and u turns about B by 2 atan(|t|) per step."""
    import torch
    tr, _, x0, u0, B, qm, dt, n_steps = _boris_case()
    x = torch.from_numpy(x0.copy()).cuda()
    u = torch.from_numpy(u0.copy()).cuda()
    xs, us = [], []
    for _ in range(n_steps // 50):
        xo, uo = rd.rd_push_boris(x, u, 50, dt, B, qm)
        xs.append(xo.cpu().numpy())
        us.append(uo.cpu().numpy())
    X, U = np.concatenate(xs, axis=1), np.concatenate(us, axis=1)
    assert np.max(np.abs(X - tr.x[:, 1:])) <= 1e-12 * np.max(np.abs(tr.x))
    assert np.max(np.abs(U - tr.u[:, 1:])) <= 1e-12 * np.max(np.abs(tr.u))
    g = np.sqrt(1.0 + np.sum(u0 * u0, axis=1))
    phi = 2.0 * np.arctan(0.5 * abs(qm) * dt * np.linalg.norm(B) / g)
    ang = np.unwrap(np.arctan2(U[:, :, 1], U[:, :, 0]), axis=1)
    assert np.max(np.abs(np.abs(ang[:, -1] - ang[:, 0]) - (n_steps - 1) * phi)) < 1e-10
    assert np.max(np.abs(np.linalg.norm(U, axis=2) - np.linalg.norm(u0, axis=1)[:, None])) < 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_runtime_coupling_push_then_deposit(precision, tol):
    """The run-time mode of Section 3.1: every 50 Boris steps on the device, the new samples are
    deposited at once by rd_deposit_stream (the first call carries the initial state as sample 0).
    Against the oracle's deposit of the numpy Boris trajectory, every cell."""
    import torch
    tr, det, x0, u0, B, qm, dt, n_steps = _boris_case()
    d = rd.RadiationDetector.from_workload(det, precision)
    x = torch.from_numpy(x0.copy()).cuda()
    u = torch.from_numpy(u0.copy()).cuda()
    q = torch.from_numpy(tr.q).cuda()
    for c in range(n_steps // 50):
        xo, uo = rd.rd_push_boris(x, u, 50, dt, B, qm)
        if c == 0:
            xo = torch.cat([torch.from_numpy(x0).cuda()[:, None], xo], dim=1).contiguous()
            uo = torch.cat([torch.from_numpy(u0).cuda()[:, None], uo], dim=1).contiguous()
            d.deposit_stream(xo, uo, q, tr.t0, dt)
        else:
            d.deposit_stream(xo, uo, q, tr.t0 + (50 * c + 1) * dt, dt)
    E, B_ = d.read()
    d.close()
    Eo, Bo, clipped = oracle.deposit(tr, det)
    assert clipped == 0
    assert parity_err(E, Eo) <= tol and parity_err(B_, Bo) <= tol
