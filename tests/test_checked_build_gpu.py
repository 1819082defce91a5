"""The checked build (RD_CHECK=1): every reduction of the mixed walk that the window margin keeps
inside the detector row verifies its bin and latches RD_ERR_BOUNDS instead of writing outside.
The library is compiled with the flag into a scratch directory and the workloads run against it in
a subprocess (a process loads one build): no bounds error, and the oracle's result."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
import oracle
import paper_2302_14812_gb300 as rd
from paper_2302_14812_gb300 import workloads as W
from parity import parity_err
rd.load_library()
oracle.build()

def multi_edge_case():
    # relativistic oscillators seen along their axis with bins 1.2 dt wide: about 8 % of the
    # (cell, interval) pairs pass two or more bin edges; cells 256-511 have shifted time origins, so
    # the window cuts their arrivals (clip tracking), cells 0-255 do not
    tr = W.oscillator_ensemble(6, 900, amp_range=(0.5, 1.0), seed=11)
    rng = np.random.default_rng(11)
    n = 512
    sgn = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    pos = np.stack([50.0 * sgn, rng.uniform(-5, 5, n), rng.uniform(-5, 5, n)], axis=1)
    shift = np.where(np.arange(n) < 256, 0.0, np.where(np.arange(n) % 4 < 2, 20.0, -20.0))
    return tr, W.Detector(pos, shift, 30.0, 1.2 * tr.dt, 1161)

cases = [("circular", *W.config_circular(), None),
         ("undulator", *W.config_undulator(n_part=8), np.array([0, 8127, 8256, 16383], dtype=np.int32)),
         ("plasma_mirror", *W.config_plasma_mirror(n_part=100_000, n_side=48, particles=slice(0, 60)),
          np.array([0, 1000, 2303], dtype=np.int32)),
         ("several_bins", *multi_edge_case(), None)]
for name, tr, det, sel in cases:
    for shape in ((256, 2), (64, 1)):
        d = rd.RadiationDetector.from_workload(det, "mixed")
        d.set_shape(shape[0], shape[1], 0, 0)
        d.deposit(torch.from_numpy(tr.x).cuda(), torch.from_numpy(tr.u).cuda(), torch.from_numpy(tr.q).cuda(),
                  tr.t0, tr.dt)
        E, B = d.read()
        st = d.stats()
        d.close()
        assert st.device_errors == 0, (name, shape, st.device_errors)
        Eo, Bo, _ = oracle.deposit(tr, det, sel)
        if sel is not None:
            E, B = E[sel], B[sel]
        err = max(parity_err(E, Eo), parity_err(B, Bo))
        assert err <= 1e-4, (name, shape, err)
        print(name, shape, "ok", err)
print("checked build ok")
"""


def test_checked_build_runs_clean(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    from paper_2302_14812_gb300 import build as B
    lib = B.build(out_dir=str(tmp_path / "checked"), defines=["RD_CHECK=1"])
    env = dict(os.environ, RD_LIBRARY=lib,
               PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests"), os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
