"""Checkpoint and resume through rd_read_fields / rd_write_fields: deposits add (Section 3.2), so a
run read back part-way and written into a new detector continues to the same result."""
import numpy as np
import pytest

import oracle
import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 2e-6}


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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("where", ["host", "device"])
def test_resume_from_checkpoint(precision, where):
    """Particles 0-2 and the first 120 steps of particles 3-5 go into one detector; its fields are
    read back (host float64 or device float32), written into a second detector, which then takes
    the rest (the other steps share their first sample with the checkpointed stretch).  The result
    equals one detector that took everything, and the oracle."""
    tr = W.random_smooth(6, 300, 0.03, seed=12)
    det = W.Detector(W.spherical_cap(5, 18.0, 0.5), None, 14.0, 0.02, 700)
    whole = rd.RadiationDetector.from_workload(det, precision)
    whole.deposit(*_dev(tr))
    Ew, Bw = whole.read()
    whole.close()

    first = rd.RadiationDetector.from_workload(det, precision)
    first.deposit(*_dev(tr.subset([0, 1, 2])))
    first.deposit(*_dev(tr.subset([3, 4, 5]).steps(0, 120)))
    if where == "host":
        Ec, Bc = first.read("float64", "cpu")
    else:
        Ec, Bc = first.read("float32", "cuda")
    first.close()

    second = rd.RadiationDetector.from_workload(det, precision)
    second.write(Ec, Bc)
    second.deposit(*_dev(tr.subset([3, 4, 5]).steps(120, 300)))
    E, B = second.read()
    st = second.stats()
    second.close()
    assert st.device_errors == 0
    tol = TOL[precision] if where == "host" or precision == "mixed" else 1e-6   # float32 checkpoint of FP64
    assert parity_err(E, Ew) <= tol and parity_err(B, Bw) <= tol
    Eo, Bo, _ = oracle.deposit(tr, det)
    bar = 1e-10 if precision == "fp64" and where == "host" else 1e-4
    assert parity_err(E, Eo) <= bar and parity_err(B, Bo) <= bar


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_write_read_round_trip_and_zero(precision):
    """write() then read() returns the written fields (exactly in the detector's precision); a None
    part is set to zero."""
    det = W.Detector(W.spherical_cap(3, 10.0, 0.3), None, 8.0, 0.05, 64)
    rng = np.random.default_rng(3)
    dt = np.float64 if precision == "fp64" else np.float32
    E = rng.normal(size=(det.n_pix, det.n_bins, 3)).astype(dt)
    B = rng.normal(size=(det.n_pix, det.n_bins, 3)).astype(dt)
    d = rd.RadiationDetector.from_workload(det, precision)
    d.write(E, B)
    Er, Br = d.read("float64", "cpu")
    assert np.array_equal(Er, E.astype(np.float64)) and np.array_equal(Br, B.astype(np.float64))
    d.write(None, B)
    Er, Br = d.read("float64", "cpu")
    assert not Er.any() and np.array_equal(Br, B.astype(np.float64))
    d.close()
