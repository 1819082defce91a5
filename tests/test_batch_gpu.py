"""Batched persistent deposit (one launch, CUDA graph) against separate deposits and the oracle.

Separate and batched deposits run the same arithmetic per work item; only the order in which FP32
reductions reach each bin differs, so they agree to ~1e-6.  Against the FP64 oracle the bar is
the mixed path's 1e-4 relative L2.
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


def _dev(tr):
    import torch
    return (torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
            tr.t0, tr.dt)


def small_problems(seed=3):
    """Six uneven problems of the three kinds."""
    probs = []
    rng = np.random.default_rng(seed)
    probs.append(W.config_undulator(n_part=7, n_steps=900, n_side=16, n_bins=256, seed=1))
    probs.append(W.config_undulator(n_part=2, n_steps=300, n_side=9, n_bins=128, gamma=8.0, seed=2))
    tr = W.circular_ensemble(5, 700, gamma=3.0, seed=4)
    pos = W.spherical_cap(12, 1e3, 0.6)
    span = 700 * tr.dt + 2.0
    probs.append((tr, W.Detector(pos, None, 1e3 - 1.0 - 0.02 * span, 1.04 * span / 300, 300)))
    tr = W.oscillator_ensemble(11, 1300, seed=5)
    pos = W.spherical_cap(8, 1e3, 0.8, axis=1)
    span = 1300 * tr.dt + 6.0
    probs.append((tr, W.Detector(pos, None, 1e3 - 3.0 - 0.02 * span, 1.04 * span / 512, 512)))
    tr = W.random_smooth(3, 250, 0.03, max_u=2.0, seed=6)
    pos = rng.normal(size=(300, 3)) * 20.0
    probs.append((tr, W.Detector(pos, rng.uniform(-1, 1, 300), 8.0, 0.03, 700)))
    probs.append(W.config_undulator(n_part=1, n_steps=64, n_side=4, n_bins=64, seed=9))
    return probs


def run_separate(probs):
    out = []
    for tr, det in probs:
        d = rd.RadiationDetector.from_workload(det, "mixed")
        d.deposit(*_dev(tr))
        out.append(d.read())
        d.close()
    return out


def run_batch(probs, stream, repeats=1):
    import torch
    dets = [rd.RadiationDetector.from_workload(det, "mixed") for _, det in probs]
    trajs = [_dev(tr) for tr, _ in probs]
    results = []
    with torch.cuda.stream(stream) if stream is not None else _null():
        for _ in range(repeats):
            for d in dets:
                d.zero(stream)
            keep = rd.deposit_batch(dets, trajs, stream)
            results.append([d.read(stream=stream) for d in dets])
            del keep
    for d in dets:
        d.close()
    return results


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


@pytest.mark.parametrize("side_stream", [True, False])
def test_batch_equals_separate_and_oracle(side_stream):
    import torch
    probs = small_problems()
    sep = run_separate(probs)
    stream = torch.cuda.Stream() if side_stream else None
    res = run_batch(probs, stream, repeats=2)
    for rep in res:
        for (E, B), (Es, Bs) in zip(rep, sep):
            assert parity_err(E, Es) <= 2e-6 and parity_err(B, Bs) <= 2e-6
    # oracle on sampled cells of every problem
    rng = np.random.default_rng(0)
    for (tr, det), (E, B) in zip(probs, res[0]):
        sel = np.sort(rng.choice(det.n_pix, size=min(4, det.n_pix), replace=False)).astype(np.int32)
        Eo, Bo, _ = oracle.deposit(tr, det, sel)
        assert parity_err(E[sel], Eo) <= 1e-4 and parity_err(B[sel], Bo) <= 1e-4


def test_batch_with_empty_problem_and_accumulation():
    import torch
    probs = small_problems()[:3]
    empty = W.Trajectories(np.zeros((0, 5, 3)), np.zeros((0, 5, 3)), np.zeros(0), 0.0, 0.1)
    probs.append((empty, probs[0][1]))
    stream = torch.cuda.Stream()
    dets = [rd.RadiationDetector.from_workload(det, "mixed") for _, det in probs]
    trajs = [_dev(tr) if tr.n_part else (torch.zeros((0, 5, 3), dtype=torch.float64, device="cuda"),
                                          torch.zeros((0, 5, 3), dtype=torch.float64, device="cuda"), None, 0.0, 0.1)
             for tr, _ in probs]
    with torch.cuda.stream(stream):
        keep = rd.deposit_batch(dets, trajs, stream)
        once = [d.read(stream=stream) for d in dets]
        keep2 = rd.deposit_batch(dets, trajs, stream)          # replayed graph, accumulates
        twice = [d.read(stream=stream) for d in dets]
    del keep, keep2
    for (E1, _), (E2, _) in zip(once[:3], twice[:3]):
        assert parity_err(E2, 2 * E1) <= 2e-6
    assert np.all(once[3][0] == 0)
    for d in dets:
        d.close()


def test_autotune_picks_a_chunk_and_result_stays_correct():
    tr, det = W.config_undulator(n_part=16, n_steps=1500, n_side=16, n_bins=512, seed=3)
    d = rd.RadiationDetector.from_workload(det, "mixed")
    chunk = d.autotune(*_dev(tr))
    assert chunk in (64, 128, 256, 512, 1024, 1500)
    E0, _ = d.read()
    assert np.all(E0 == 0)                                   # autotuning leaves zeroed fields
    d.deposit(*_dev(tr))
    E, B = d.read()
    sel = np.array([0, 100, 255], dtype=np.int32)
    Eo, Bo, _ = oracle.deposit(tr, det, sel)
    assert parity_err(E[sel], Eo) <= 1e-4
    d.close()


def test_uneven_64_problem_set_reduced_particles():
    """The 64 uneven problems (undulator / circular / oscillator, steps 500-8000, 32^2-128^2 cells,
    16*side bins) with particle counts scaled by 0.004: one batched launch vs separate launches
    (compared on the device, problem by problem), and the oracle on one cell of every eighth
    problem.  The batched launch takes one batch-wide step chunk (halved while the batch is short of
    work items) while a separate launch of a small problem halves its chunk to fill the GPU, so the
    two FP32 walks re-anchor at different steps and agree to the mixed path's rounding (bar 1e-5,
    ten times below the oracle bar), not bit for bit."""
    import torch
    probs = [(tr, det) for _, tr, det in W.batch_problems(64, seed=4, scale=0.004)]
    stream = torch.cuda.Stream()
    dets = [rd.RadiationDetector.from_workload(det, "mixed") for _, det in probs]
    trajs = [_dev(tr) for tr, _ in probs]
    with torch.cuda.stream(stream):
        keep = rd.deposit_batch(dets, trajs, stream)
        stream.synchronize()
    for i, (tr, det) in enumerate(probs):
        Eb, Bb = dets[i].read("float32", "cuda", stream=stream)
        s = rd.RadiationDetector.from_workload(det, "mixed")
        s.deposit(*trajs[i])
        Es, Bs = s.read("float32", "cuda")
        torch.cuda.synchronize()
        for a, b in ((Eb, Es), (Bb, Bs)):
            err = float(torch.linalg.norm((a - b).double()) / max(float(torch.linalg.norm(b.double())), 1e-300))
            assert err <= 1e-5, (i, err)
        if i % 8 == 0:
            sel = np.array([det.n_pix // 2], dtype=np.int32)
            Eo, _, _ = oracle.deposit(tr, det, sel)
            assert parity_err(Eb[sel].double().cpu().numpy(), Eo) <= 1e-4
        s.close()
        del Eb, Bb, Es, Bs
    del keep
    for d in dets:
        d.close()


def test_batch_record_budget_splits_into_groups():
    """A 150 KB record budget splits the six problems into particle segments and ~20 launch groups
    (each records + one persistent launch); results equal separate deposits, on first capture and
    on replay (accumulating)."""
    import torch
    probs = small_problems()
    sep = run_separate(probs)
    stream = torch.cuda.Stream()
    dets = [rd.RadiationDetector.from_workload(det, "mixed") for _, det in probs]
    dets[0].set_batch_budget(150_000)
    trajs = [_dev(tr) for tr, _ in probs]
    with torch.cuda.stream(stream):
        keep = rd.deposit_batch(dets, trajs, stream)
        once = [d.read(stream=stream) for d in dets]
        keep2 = rd.deposit_batch(dets, trajs, stream)          # replayed graph, accumulates
        twice = [d.read(stream=stream) for d in dets]
    del keep, keep2
    for (E, B), (E2, B2), (Es, Bs) in zip(once, twice, sep):
        assert parity_err(E, Es) <= 2e-6 and parity_err(B, Bs) <= 2e-6
        assert parity_err(E2, 2 * Es) <= 2e-6 and parity_err(B2, 2 * Bs) <= 2e-6
    dets[0].set_batch_budget(0)                                   # back to the default: one group
    for d in dets:
        d.zero(stream)
    with torch.cuda.stream(stream):
        keep = rd.deposit_batch(dets, trajs, stream)
        again = [d.read(stream=stream) for d in dets]
    del keep
    for (E, B), (Es, Bs) in zip(again, sep):
        assert parity_err(E, Es) <= 2e-6 and parity_err(B, Bs) <= 2e-6
    for d in dets:
        d.close()


def test_batch_mixes_modes():
    """One batch with a linear-interpolation problem, a far-field problem and a plain one (three walk
    families, so three persistent launches in the batch's graph) equals the separate deposits."""
    import torch
    probs = small_problems()[:3]
    probs[0][1].flags = W.RD_NEAR | W.RD_FAR | W.RD_LINEAR
    probs[1][1].flags = W.RD_FAR | W.RD_FARFIELD
    sep = run_separate(probs)
    res = run_batch(probs, torch.cuda.Stream())
    for (E, B), (Es, Bs) in zip(res[0], sep):
        assert parity_err(E, Es) <= 2e-6 and parity_err(B, Bs) <= 2e-6


def test_uneven_64_problem_set_full_scale():
    """The 64 uneven problems at their stated size (particle counts log-uniform in [100, 5e4], steps
    500-8000, 32^2-128^2 cells x 16*side bins; ~1e13 deposits, ~1e11 FP64 trajectory values
    generated on the device) in one rd_deposit_batch call (records in launch groups of at most
    4 GiB); 16 random cells of every problem against the FP64 oracle at the mixed bar."""
    import torch
    probs = W.batch_problems_torch(64, seed=4, scale=1.0)
    stream = torch.cuda.Stream()
    dets = [rd.RadiationDetector.from_workload(det, "mixed") for _, _, det in probs]
    trajs = [t for _, t, _ in probs]
    with torch.cuda.stream(stream):
        keep = rd.deposit_batch(dets, trajs, stream)
        stream.synchronize()
    del keep
    rng = np.random.default_rng(44)
    worst = 0.0
    for i in range(len(probs)):
        kind, (x, u, q, t0, dt), det = probs[i]
        sel = np.sort(rng.choice(det.n_pix, 16, replace=False)).astype(np.int32)
        E, B = dets[i].read("float32", "cuda", stream=stream)
        stream.synchronize()
        idx = torch.from_numpy(sel.astype(np.int64)).cuda()
        Eb, Bb = E[idx].double().cpu().numpy(), B[idx].double().cpu().numpy()
        st = dets[i].stats()
        dets[i].close()
        del E, B
        tr = W.Trajectories(x.cpu().numpy(), u.cpu().numpy(), q.cpu().numpy(), t0, dt)
        probs[i] = None
        trajs[i] = None
        del x, u, q
        assert st.device_errors == 0, (i, kind)
        Eo, Bo, _ = oracle.deposit(tr, det, sel)
        err = max(parity_err(Eb, Eo), parity_err(Bb, Bo))
        worst = max(worst, err)
        assert err <= 1e-4, (i, kind, err)
    print(f"64 problems at full scale: worst parity error {worst:.3e}")
