"""The multi-rank (torchrun) host path of the benchmark, on CPU with the gloo backend.

Each rank runs its own independent ensemble (weak scaling): ranks must get distinct seeds of the
same workload shape, agree on the slowest rank's time, and report the whole-job throughput.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2302_14812_gb300 import workloads as W
    tr, det = W.config_undulator(n_part=3, n_steps=40, n_side=4, n_bins=64, seed=bench.rank_seed(rank))
    my_ms = 10.0 + 5.0 * rank
    slow = bench.max_over_ranks(my_ms, dist, "cpu")
    value = bench.job_throughput(W.deposits(tr, det), world, slow)
    out.put((rank, float(tr.x[0, 5, 1]), slow, value, W.deposits(tr, det)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, y0, s0, v0, d0), (r1, y1, s1, v1, d1) = res
    assert y0 != y1                         # independent ensembles
    assert d0 == d1                         # same shape per rank
    assert s0 == s1 == 15.0                 # both ranks report the slowest time
    assert v0 == v1 == pytest.approx(2 * d0 / 0.015)
