#!/usr/bin/env python3
"""Throughput of the radiation deposit on one GB300: particle*step*cell deposits per second.

Workload (default): the planar-undulator ensemble -- 1000 electrons (gamma 20, K 1, 10 periods,
seeded phases and offsets) x 4000 steps, spherical cap of 128x128 cells at 1e4 periods,
2048 time bins per cell (6.55e10 deposits per step).  A step = one full deposit of that
workload into a zeroed detector (per-sample precompute + deposit kernel).

Arms:
  default            mixed-precision path (FP32 fields/accumulation, FP64-anchored arrival times),
                     also timing the plain FP64 GPU path and the FP64 CPU oracle on a sample
  --impl reference   the FP64 CPU oracle alone (the method as the paper defines it), on the
                     host cores, each step a bounded sample (a subset of cells, all particles)

Multi-GPU (torchrun): every rank deposits its own independent ensemble (weak scaling, no data
exchange); ranks meet only at the timing barriers and the max-over-ranks time reduction.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle·step·pixel deposits/sec, FP32-mixed vs FP64 on one GB300 at ≤1e-4 rel L2"
UNIT = "deposits/s"
# FP32 operations of the mixed kernel, counted from its source (add/sub/mul = 1, fused
# multiply-add = 2; the 3 MUFU reciprocal / reciprocal-square-root ops are not counted):
#   per deposit: geometry and Eq. 1 with B = n x E and the arrival-time increment 58,
#                integrating accumulation into the running bin 17
#   per bin edge crossed: starting the next bin with the rest of the interval 9
FLOPS_PER_DEPOSIT_MIXED = 75
FLOPS_PER_CROSSING_MIXED = 9
# FP64 operations of the plain kernel per deposit, counted from its source the same way (square
# root, reciprocal and the bin-edge compare count 1 each): arrival time (Eq. 2, t_k from the record)
# 12, Eq. 1 multiplied out over the one reciprocal 1/(kappa R) with B = n x E (charge folded into
# the record) 44, accumulation into the running bin 14.
FLOPS_PER_DEPOSIT_FP64 = 70
# FP32 lanes per multiprocessor of this architecture (sm_103a: 4 sub-partitions x 32).
FP32_LANES_PER_SM = 128
WORKLOAD_UNDULATOR = ("undulator ensemble: 1000 e- (gamma 20, K 1, 10 periods) x 4000 steps, "
                      "128x128-cell spherical cap at 1e4 periods x 2048 bins")


def undulator_workload(n_part: int) -> str:
    """Workload name of the undulator ensemble with n_part electrons (the headline has 1000)."""
    return WORKLOAD_UNDULATOR.replace("1000 e-", f"{n_part} e-", 1)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "deposit_mixed_undulator_ncu.md")
# the headline kernel and the files that fix its launch (work items, step chunk, shapes): the
# committed traffic figure holds only for the revision it was captured on
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2302_14812_gb300", "csrc", f)
                  for f in ("rd_mixed.cu", "rd_internal.cuh", "rd_api.cu")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--particles", type=int, default=1000)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-farfield", action="store_true", help="skip the far-field-limit leg")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the linear-interpolation, streaming and spectrum legs")
    ap.add_argument("--workload", choices=["undulator", "batch", "adjoint", "plasma_mirror"], default="undulator",
                    help="undulator: the headline deposit; batch: 64 uneven problems, one persistent "
                         "launch vs separate launches; adjoint: gradient kernel")
    ap.add_argument("--pm-particles", type=int, default=100_000,
                    help="electrons of the plasma-mirror workload (1e5 = the full configuration)")
    ap.add_argument("--pm-chunk", type=int, default=10_000, help="electrons generated and deposited per chunk")
    ap.add_argument("--adjoint-particles", type=int, default=10_000,
                    help="electrons of the adjoint workload (1e4 = the full configuration)")
    ap.add_argument("--adjoint-fp64-particles", type=int, default=100,
                    help="electrons of the adjoint workload given to the FP64 adjoint (0 = skip that leg)")
    ap.add_argument("--shape", default=None,
                    help="deposit shape of the mixed detector as CELLSxPER_THREAD[xCHUNKxGROUP] (default: the "
                         "library's automatic shape)")
    ap.add_argument("--batch-scale", type=float, default=0.1,
                    help="particle-count scale of the 64-problem set (memory: every problem resident)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(rank: int) -> int:
    """Seed of rank r's independent ensemble (weak scaling: same shape, different particles)."""
    return 2 + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The slowest rank's time (host-side timing reduction, not a data-path collective)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(deposits_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job deposits/s: every rank processes deposits_per_rank per step."""
    return deposits_per_rank * world / (ms_per_step / 1e3)


# ----------------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: RD_CLOCKS_CSV if set (a per-rank suffix is added), else a temporary file
        base = os.environ.get("RD_CLOCKS_CSV")
        self.path = (f"{base}.rank{gpu_index}" if base else f"/tmp/rd_clocks_{os.getpid()}_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        # the timed region starts once the sampler has written its first sample: its start-up
        # (attaching to the driver) then does not fall inside the region
        t_end = time.perf_counter() + 5.0
        while time.perf_counter() < t_end and self.proc.poll() is None:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                pass
            time.sleep(0.02)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        mx = np.array([num(r[2]) for r in rows])
        pw = np.array([num(r[3]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_min_mhz": float(np.nanmin(sm)), "sm_max_mhz": float(np.nanmax(mx)),
                "power_w_max": float(np.nanmax(pw)), "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------------------------
def profile_traffic():
    """DRAM bytes per launch of the mixed deposit kernel from the committed ncu summary, if the
    summary was taken on the current kernel and launch sources (else None)."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
    if not m or not h:
        return None
    return float(m.group(1)) if h.group(1) == kernel_sources_sha() else None


def kernel_sources_sha() -> str:
    """sha256 over the concatenated KERNEL_SOURCES."""
    sha = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            sha.update(fh.read())
    return sha.hexdigest()


def fp32_peak(sm_mhz):
    """(TFLOP/s, description): FP32 FMA peak derived from this device's multiprocessor count, its
    FP32 lanes and the median SM clock sampled during the timed region (max clock if none)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, src = sm_mhz, "median SM clock sampled during the timed region"
    if not mhz or not math.isfinite(mhz):
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz, src = float(json.load(f)["sm_max_mhz"]), "maximum SM clock of this pool's GPUs"
        except (OSError, KeyError, ValueError):
            mhz, src = 2070.0, "nominal maximum SM clock"
    tf = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return tf, f"derived: {sms} SM x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz ({src})"


def hbm_peak():
    """(GB/s, kind): the measured copy bandwidth of this machine's GPUs if recorded, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_link_gbs(host_out, host_in, reps: int = 3):
    """Plain copy rates between pinned host memory and the device (GB/s), for reading the e2e number:
    the readback of one field array (device -> host) and the upload of the positions (host -> device)."""
    import torch
    dev_out = torch.empty(host_out.shape, dtype=host_out.dtype, device="cuda")
    dev_in = torch.empty(host_in.shape, dtype=host_in.dtype, device="cuda")
    rates = {}
    for name, dst, src in (("d2h_gbs", host_out, dev_out), ("h2d_gbs", dev_in, host_in)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        rates[name] = reps * src.numel() * src.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9
    del dev_out, dev_in
    return rates


def oracle_rate(tr, det, target_s: float, sel_seed: int = 0):
    """Run the oracle on a bounded sample of cells (all particles and steps); returns
    (deposits/s, seconds, n_cells, threads, sel)."""
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    rng = np.random.default_rng(sel_seed)
    # calibration: one cell per thread
    n_cal = min(det.n_pix, threads)
    sel = rng.choice(det.n_pix, size=n_cal, replace=False).astype(np.int32)
    t = time.perf_counter()
    oracle.deposit(tr, det, sel, threads)
    dt_cal = time.perf_counter() - t
    n_cells = int(min(det.n_pix, max(n_cal, n_cal * math.floor(target_s / max(dt_cal, 1e-3)))))
    sel = rng.choice(det.n_pix, size=n_cells, replace=False).astype(np.int32)
    t = time.perf_counter()
    E, B, _ = oracle.deposit(tr, det, sel, threads)
    secs = time.perf_counter() - t
    dep = tr.n_part * tr.n_steps * n_cells
    return dep / secs, secs, n_cells, threads, sel, E, B


def run_reference(args, rank, world):
    """FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    from paper_2302_14812_gb300 import workloads as W
    tr, det = W.config_undulator(n_part=args.particles)
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    total = max(1, args.steps + args.warmup)
    per_step = max(5.0, min(30.0, 150.0 / total))
    rng = np.random.default_rng(1)
    # calibrate cells per step
    sel = rng.choice(det.n_pix, size=threads, replace=False).astype(np.int32)
    t = time.perf_counter()
    oracle.deposit(tr, det, sel, threads)
    dt_cal = time.perf_counter() - t
    n_cells = int(min(det.n_pix, max(threads, threads * math.floor(per_step / max(dt_cal, 1e-3)))))
    for _ in range(args.warmup):
        oracle.deposit(tr, det, rng.choice(det.n_pix, size=n_cells, replace=False).astype(np.int32), threads)
    secs = 0.0
    for _ in range(args.steps):
        s = rng.choice(det.n_pix, size=n_cells, replace=False).astype(np.int32)
        t = time.perf_counter()
        oracle.deposit(tr, det, s, threads)
        secs += time.perf_counter() - t
    dep = tr.n_part * tr.n_steps * n_cells
    value = dep * args.steps / secs
    sample = (f"{n_cells} random cells of 16384 x all {tr.n_part} particles x {tr.n_steps} steps "
              f"per step ({dep:.3g} deposits)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": undulator_workload(tr.n_part), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
def run_batch_workload(args):
    """64 uneven problems: one rd_deposit_batch (persistent kernel, graph replay) against 64
    separate rd_deposit_trajectories calls on the same stream."""
    import torch
    import paper_2302_14812_gb300 as rd
    from paper_2302_14812_gb300 import workloads as W
    rd.load_library()
    # the trajectories are generated on the device (at full scale they hold ~1e11 FP64 values)
    probs = W.batch_problems_torch(64, seed=4, scale=args.batch_scale)
    stream = torch.cuda.Stream()
    dets, trajs, deposits = [], [], 0
    for _, t, det in probs:
        dets.append(rd.RadiationDetector.from_workload(det, "mixed", stream))
        trajs.append(t)
        deposits += t[0].shape[0] * (t[0].shape[1] - 1) * det.n_pix
    del probs
    torch.cuda.synchronize()

    def separate():
        for d, t in zip(dets, trajs):
            d.deposit(*t, stream=stream)

    def batched():
        rd.deposit_batch(dets, trajs, stream)

    out = {}
    with torch.cuda.stream(stream):
        for name, fn in (("separate", separate), ("batch", batched)):
            for _ in range(args.warmup):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            out[name] = {"ms_per_step": ms, "value": deposits / (ms / 1e3)}
    for d in dets:
        d.close()
    line = {"metric": "deposits/sec, 64 uneven problems in one persistent launch (CUDA graph)",
            "value": out["batch"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["batch"]["ms_per_step"], "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"64 problems (undulator/circular/oscillator, particles log-uniform "
                                   f"[100,5e4] x {args.batch_scale}, steps 500-8000, 32^2..128^2 cells x "
                                   f"16*side bins)", "deposits_per_step": deposits},
            "separate_launches": out["separate"],
            "speedup_batch_vs_separate": out["separate"]["ms_per_step"] / out["batch"]["ms_per_step"]}
    print(json.dumps(line), flush=True)


def run_adjoint_workload(args):
    """Forward and adjoint of 1e4 undulator electrons (gamma 10) x 2000 steps on 64x64 x 1024."""
    import torch
    import paper_2302_14812_gb300 as rd
    from paper_2302_14812_gb300 import workloads as W
    rd.load_library()
    tr, det = W.config_undulator(n_part=args.adjoint_particles, n_steps=2000, n_side=64, n_bins=1024, gamma=10.0,
                                 K=1.0, n_periods=10.0, distance=1e4, seed=5)
    deposits = W.deposits(tr, det)
    x = torch.from_numpy(tr.x).cuda()
    u = torch.from_numpy(tr.u).cuda()
    q = torch.from_numpy(tr.q).cuda()
    d = rd.RadiationDetector.from_workload(det, "mixed")
    d.set_timing(True)
    # loss 1/2 sum |E - E_target|^2 over E: the target is the deposit of the same electrons with
    # seeded perturbations of 1e-4 (a position offset and a momentum scale per electron), and the
    # adjoint's input is the misfit E - E_target
    rng = np.random.default_rng(5)
    x_off = torch.from_numpy(1e-4 * rng.normal(size=(tr.n_part, 1, 3))).cuda()
    u_scl = torch.from_numpy(1.0 + 1e-4 * rng.normal(size=(tr.n_part, 1, 1))).cuda()
    d.deposit(x + x_off, u * u_scl, q, tr.t0, tr.dt)
    E_tgt, _ = d.read("float32", "cuda")
    d.zero()
    d.deposit(x, u, q, tr.t0, tr.dt)
    gE, _ = d.read("float32", "cuda")
    gE -= E_tgt
    misfit_rel = float(torch.linalg.norm(gE) / torch.linalg.norm(E_tgt))
    del E_tgt, x_off, u_scl
    dc = rd.RadiationDetector.from_workload(det, "mixed")
    dc.set_timing(True)
    dc.set_adjoint_mode("compensated")
    res = {}
    for name in ("forward", "adjoint", "adjoint_compensated"):
        dd = dc if name == "adjoint_compensated" else d

        def step():
            if name == "forward":
                d.zero()
                d.deposit(x, u, q, tr.t0, tr.dt)
            else:
                dd.adjoint(x, u, q, tr.t0, tr.dt, gE)
        for _ in range(args.warmup):
            step()
        dd.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        st = dd.stats()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms_per_step": ms, "value": deposits / (ms / 1e3),
                     "kernel_ms": st.kernel_ms / max(1, st.kernel_launches)}

    # the plain FP64 adjoint on the first particles of the same workload, and the two adjoints'
    # agreement there
    fp64 = None
    n64 = min(args.adjoint_fp64_particles, tr.n_part)
    if n64 > 0:
        sub = tr.subset(list(range(n64)))
        x64, u64, q64 = (torch.from_numpy(a).cuda() for a in (sub.x, sub.u, sub.q))
        d64 = rd.RadiationDetector.from_workload(det, "fp64")
        d64.adjoint(x64, u64, q64, sub.t0, sub.dt, gE)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gx64, gu64 = d64.adjoint(x64, u64, q64, sub.t0, sub.dt, gE)
        e1.record()
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        gxm, gum = d.adjoint(x64, u64, q64, sub.t0, sub.dt, gE)
        gxc, guc = dc.adjoint(x64, u64, q64, sub.t0, sub.dt, gE)
        torch.cuda.synchronize()
        rate64 = W.deposits(sub, det) / (ms64 / 1e3)

        def rel(a, b):
            return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        fp64 = {"particles": n64, "ms_per_step": ms64, "value": rate64,
                "mixed_speedup": res["adjoint"]["value"] / rate64,
                "compensated_speedup": res["adjoint_compensated"]["value"] / rate64,
                "mixed_vs_fp64_rel_l2": {"x": rel(gxm, gx64), "u": rel(gum, gu64)},
                "compensated_vs_fp64_rel_l2": {"x": rel(gxc, gx64), "u": rel(guc, gu64)}}
        d64.close()
    d.close()
    dc.close()
    line = {"metric": "deposits/sec of the adjoint (gather) kernel, gradient wrt positions and momenta",
            "value": res["adjoint"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["adjoint"]["ms_per_step"], "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{tr.n_part} undulator e- (gamma 10, K 1) x 2000 steps, 64x64 cap x 1024 "
                                   "bins, anchors recomputed every 250 samples; loss 1/2 |E - E_target|^2, target "
                                   "from trajectories perturbed by 1e-4", "deposits_per_step": deposits,
                       "misfit_rel_l2": misfit_rel},
            "forward": res["forward"], "adjoint": res["adjoint"],
            "adjoint_compensated": res["adjoint_compensated"], "fp64_adjoint": fp64,
            "adjoint_over_forward_time": res["adjoint"]["ms_per_step"] / res["forward"]["ms_per_step"]}
    print(json.dumps(line), flush=True)


def run_plasma_mirror_workload(args):
    """The plasma-mirror configuration at full size: 1e5 electrons x 10000 steps onto 256x256 cells
    x 4096 bins (6.55e13 deposits), generated on the device in particle chunks and deposited
    (accumulating) into one mixed detector; the FP64 GPU path on 64 random cells of the same
    detector and the CPU oracle on 2 of them give the parity of the full-size result."""
    import torch
    import oracle
    import paper_2302_14812_gb300 as rd
    from paper_2302_14812_gb300 import workloads as W
    rd.load_library()
    oracle.build()
    n_part, n_steps = args.pm_particles, 10_000
    dt = 12.0 * 2.0 * math.pi / n_steps
    det = W.plasma_mirror_detector(dt)
    rng = np.random.default_rng(3)
    cells64 = np.sort(rng.choice(det.n_pix, 64, replace=False))
    sel2 = np.sort(rng.choice(64, 2, replace=False)).astype(np.int32)
    sub = det.subset(cells64)
    dm = rd.RadiationDetector.from_workload(det, "mixed")
    d64 = rd.RadiationDetector.from_workload(sub, "fp64")
    Eo = np.zeros((2, det.n_bins, 3))
    Bo = np.zeros((2, det.n_bins, 3))
    t_mixed = t_fp64 = t_oracle = 0.0
    for p0 in range(0, n_part, args.pm_chunk):
        x, u, q, (t0, dtc) = W.plasma_mirror_surface_torch(slice(p0, min(n_part, p0 + args.pm_chunk)),
                                                           n_part=n_part, n_steps=n_steps)
        torch.cuda.synchronize()
        for d, which in ((dm, "mixed"), (d64, "fp64")):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            d.deposit(x, u, q, t0, dtc)
            e1.record()
            e1.synchronize()
            if which == "mixed":
                t_mixed += e0.elapsed_time(e1) / 1e3
            else:
                t_fp64 += e0.elapsed_time(e1) / 1e3
        tr = W.Trajectories(x.cpu().numpy(), u.cpu().numpy(), q.cpu().numpy(), t0, dtc)
        c0 = time.perf_counter()
        e_o, b_o, _ = oracle.deposit(tr, sub, sel2)
        t_oracle += time.perf_counter() - c0
        Eo += e_o
        Bo += b_o
        del x, u, q, tr
    E, B = dm.read("float32", "cuda")
    idx = torch.from_numpy(cells64).cuda()
    Em, Bm = E[idx].double().cpu().numpy(), B[idx].double().cpu().numpy()
    del E, B
    E64, B64 = d64.read()
    st = dm.stats()
    dm.close()
    d64.close()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    deposits = n_part * n_steps * det.n_pix
    line = {"metric": "particle·step·pixel deposits/sec, plasma-mirror configuration at full size",
            "value": deposits / t_mixed, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (generated on the device in particle chunks)",
            "config": {"workload": f"plasma-mirror surface: {n_part} e- (a0 5, 20 harmonics n^-2, 12 periods) x "
                                   f"{n_steps} steps, 256x256-cell plane x 4096 bins", "deposits": deposits,
                       "particle_chunk": args.pm_chunk},
            "seconds_mixed": t_mixed, "bin_crossings": st.n_bin_crossings, "clipped": st.n_clipped,
            "fp64_gpu_64_cells": {"value": n_part * n_steps * 64 / t_fp64, "seconds": t_fp64},
            "parity": {"mixed_vs_fp64_gpu_64_cells_E": rel(Em, E64), "mixed_vs_fp64_gpu_64_cells_B": rel(Bm, B64),
                       "mixed_vs_oracle_2_cells_E": rel(Em[sel2], Eo), "mixed_vs_oracle_2_cells_B": rel(Bm[sel2], Bo),
                       "fp64_gpu_vs_oracle_2_cells_E": rel(E64[sel2], Eo),
                       "fp64_gpu_vs_oracle_2_cells_B": rel(B64[sel2], Bo)},
            "oracle_2_cells": {"value": n_part * n_steps * 2 / t_oracle, "seconds": t_oracle,
                               "cores": oracle.default_threads()}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch_workload(args)
        return
    if args.workload == "adjoint":
        run_adjoint_workload(args)
        return
    if args.workload == "plasma_mirror":
        run_plasma_mirror_workload(args)
        return

    import torch
    import paper_2302_14812_gb300 as rd
    from paper_2302_14812_gb300 import workloads as W

    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    rd.load_library()

    # every rank: its own independent ensemble of the same shape (weak scaling)
    tr, det = W.config_undulator(n_part=args.particles, seed=rank_seed(rank))
    deposits = W.deposits(tr, det)
    xd = torch.from_numpy(tr.x).to(dev)
    ud = torch.from_numpy(tr.u).to(dev)
    qd = torch.from_numpy(tr.q).to(dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def slowest(v: float) -> float:
        return max_over_ranks(v, dist, dev)

    # ---------------- mixed path, inputs resident in HBM ----------------
    mixed = rd.RadiationDetector.from_workload(det, "mixed")
    if args.shape:
        mixed.set_shape(*[int(v) for v in args.shape.lower().split("x")])
    mixed.set_timing(True)
    for _ in range(args.warmup):
        mixed.zero()
        mixed.deposit(xd, ud, qd, tr.t0, tr.dt)
    mixed.stats()                      # drop warm-up kernel timings
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            mixed.zero()
            mixed.deposit(xd, ud, qd, tr.t0, tr.dt)
        ev1.record(stream)
        barrier()
    ms_total = slowest(ev0.elapsed_time(ev1))
    st = mixed.stats()
    clocks = clk.summary()
    ms_step = ms_total / args.steps
    kernel_ms = st.kernel_ms / max(1, st.kernel_launches)
    launches = 2 * args.steps          # per step: precompute + deposit kernel
    value = job_throughput(deposits, world, ms_step)

    E_mixed, B_mixed = mixed.read("float64", "cpu")
    mixed_shape = mixed.shape()

    # ---------------- plain FP64 GPU path (speedup reference) ----------------
    fp64_info = None
    if args.fp64_steps > 0:
        f64 = rd.RadiationDetector.from_workload(det, "fp64")
        f64.set_timing(True)
        f64.deposit(xd, ud, qd, tr.t0, tr.dt)
        f64.stats()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            f64.zero()
            f64.deposit(xd, ud, qd, tr.t0, tr.dt)
        e1.record(stream)
        barrier()
        ms64 = slowest(e0.elapsed_time(e1)) / args.fp64_steps
        E64, B64 = f64.read("float64", "cpu")
        rel_e = float(np.linalg.norm(E_mixed - E64) / np.linalg.norm(E64))
        rel_b = float(np.linalg.norm(B_mixed - B64) / np.linalg.norm(B64))
        fp64_info = {"value": deposits * world / (ms64 / 1e3), "ms_per_step": ms64,
                     "speedup_mixed_vs_fp64": ms64 / ms_step,
                     "mixed_rel_l2_vs_fp64_gpu": {"E": rel_e, "B": rel_b},
                     "achieved_fp64_tflops": FLOPS_PER_DEPOSIT_FP64 * deposits / (ms64 / 1e3) / 1e12,
                     "flops_per_deposit": FLOPS_PER_DEPOSIT_FP64}
        f64.close()
        del E64, B64

    # ---------------- far-field limit (RD_FARFIELD) on the same workload ----------------
    ff_info = None
    if not args.no_farfield:
        det_ff = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins, W.RD_FAR | W.RD_FARFIELD)
        ffd = rd.RadiationDetector.from_workload(det_ff, "mixed")
        for _ in range(max(1, args.warmup)):
            ffd.zero()
            ffd.deposit(xd, ud, qd, tr.t0, tr.dt)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ffd.zero()
            ffd.deposit(xd, ud, qd, tr.t0, tr.dt)
        e1.record(stream)
        barrier()
        ms_ff = slowest(e0.elapsed_time(e1)) / args.steps
        ffd.close()
        ff_info = {"value": deposits * world / (ms_ff / 1e3), "ms_per_step": ms_ff,
                   "speedup_vs_exact": ms_step / ms_ff,
                   "mode": "far-field limit: Eq. 3 arrival times, radiation term at the cell direction"}

    # ------- linear interpolation, streamed stretches and spectra on the same workload -------
    variants = None
    if not args.no_variants:
        variants = {}

        def timed(fn, n):
            for _ in range(max(1, min(args.warmup, 2))):
                fn()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            barrier()
            return slowest(e0.elapsed_time(e1)) / n

        det_lin = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins,
                             W.RD_NEAR | W.RD_FAR | W.RD_LINEAR)
        ld = rd.RadiationDetector.from_workload(det_lin, "mixed")

        def lin_step():
            ld.zero()
            ld.deposit(xd, ud, qd, tr.t0, tr.dt)
        ms_lin = timed(lin_step, 2)
        ld.close()
        variants["linear"] = {"value": deposits * world / (ms_lin / 1e3), "ms_per_step": ms_lin,
                              "vs_held": ms_step / ms_lin,
                              "mode": "RD_LINEAR: field linear in arrival time over each interval"}

        det_prev = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins,
                              W.RD_NEAR | W.RD_FAR | W.RD_HOLD_PREV)
        pd = rd.RadiationDetector.from_workload(det_prev, "mixed")

        def prev_step():
            pd.zero()
            pd.deposit(xd, ud, qd, tr.t0, tr.dt)
        ms_prev = timed(prev_step, 2)
        pd.close()
        variants["hold_prev"] = {"value": deposits * world / (ms_prev / 1e3), "ms_per_step": ms_prev,
                                 "vs_held": ms_step / ms_prev,
                                 "mode": "RD_HOLD_PREV: interval k holds the field of sample k-1"}

        det_quad = W.Detector(det.pix_pos, det.pix_t0, det.t_min, det.dt_det, det.n_bins,
                              W.RD_NEAR | W.RD_FAR | W.RD_QUADRATIC)
        qdd = rd.RadiationDetector.from_workload(det_quad, "mixed")

        def quad_step():
            qdd.zero()
            qdd.deposit(xd, ud, qd, tr.t0, tr.dt)
        ms_quad = timed(quad_step, 2)
        qdd.close()
        variants["quadratic"] = {"value": deposits * world / (ms_quad / 1e3), "ms_per_step": ms_quad,
                                 "vs_held": ms_step / ms_quad,
                                 "mode": "RD_QUADRATIC: field quadratic in arrival time through samples k-2, k-1, k"}

        n_str = 8
        bounds = np.linspace(0, tr.n_samples, n_str + 1).astype(int)
        pieces = [(xd[:, a:b].contiguous(), ud[:, a:b].contiguous(), tr.t0 + a * tr.dt)
                  for a, b in zip(bounds[:-1], bounds[1:])]
        sd = rd.RadiationDetector.from_workload(det, "mixed")

        def stream_step():
            sd.stream_reset()
            sd.zero()
            for px, pu, pt0 in pieces:
                sd.deposit_stream(px, pu, qd, pt0, tr.dt)
        ms_str = timed(stream_step, 2)
        E_str, _ = sd.read("float64", "cpu")
        sd.close()
        del pieces
        variants["stream"] = {"value": deposits * world / (ms_str / 1e3), "ms_per_step": ms_str,
                              "stretches": n_str, "vs_single_call": ms_step / ms_str,
                              "rel_l2_E_vs_single_call": float(np.linalg.norm(E_str - E_mixed) / np.linalg.norm(E_mixed)),
                              "mode": f"rd_deposit_stream: the trajectories handed over in {n_str} stretches"}
        del E_str

        ms_sp = timed(lambda: mixed.power_spectrum("E"), 3)
        nbytes = det.n_pix * det.n_bins * 32 + det.n_pix * (det.n_bins // 2 + 1) * 4
        peak, kind = hbm_peak()
        gbs = nbytes / (ms_sp / 1e3) / 1e9
        variants["spectrum"] = {"ms": ms_sp, "spectra_per_s": det.n_pix * world / (ms_sp / 1e3),
                                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                             "frac": gbs / peak, "peak_kind": kind,
                                             "bytes": nbytes,
                                             "bytes_kind": "field sectors read (32 B per bin and cell) + spectrum written"},
                                "mode": "rd_power_spectrum of E: two FP32 transforms per cell in shared memory"}

    # ---------------- end to end through the C ABI with host buffers ----------------
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(tr.x).pin_memory()
        uh = torch.from_numpy(tr.u).pin_memory()
        qh = torch.from_numpy(tr.q).pin_memory()
        Eh = torch.empty((det.n_pix, det.n_bins, 3), dtype=torch.float32).pin_memory()
        Bh = torch.empty_like(Eh).pin_memory()
        h2d = (xh.numel() + uh.numel() + qh.numel()) * 8
        d2h = (Eh.numel() + Bh.numel()) * 4

        # Three detectors on three CUDA streams.  Step i is enqueued as upload + deposit + readback
        # (asynchronous, into pinned host memory) on stream i % 3; the host then waits for step i-2
        # and checks its errors.  So the next steps' uploads run on a copy engine during step i's
        # kernel, step i's readback conversion runs before the next kernel, and its copy to the host
        # during that kernel; with two steps queued ahead, a late host wake-up does not leave the GPU
        # without work.  Every step uploads its trajectories from pinned host memory and reads its
        # fields back to the host.
        # The readback runs on a high-priority stream (after the deposit's event), so that its layout
        # conversion is dispatched ahead of the CTAs of the next step's kernel, which is already
        # queued on another stream.
        depth = 3
        streams = [torch.cuda.Stream() for _ in range(depth)]
        top = torch.cuda.Stream.priority_range()[1] if hasattr(torch.cuda.Stream, "priority_range") else -1
        rstreams = [torch.cuda.Stream(priority=top) for _ in range(depth)]
        pair = [mixed] + [rd.RadiationDetector.from_workload(det, "mixed") for _ in range(depth - 1)]
        Ehs = [Eh] + [torch.empty_like(Eh).pin_memory() for _ in range(depth - 1)]
        Bhs = [Bh] + [torch.empty_like(Bh).pin_memory() for _ in range(depth - 1)]

        def enqueue(i):
            j = i % depth
            pair[j].zero(streams[j])
            pair[j].deposit(xh, uh, qh, tr.t0, tr.dt, stream=streams[j])   # H2D inside the call
            ev = torch.cuda.Event()
            ev.record(streams[j])
            rstreams[j].wait_event(ev)
            rd.rd_read_fields(pair[j].handle, Ehs[j].data_ptr(), Bhs[j].data_ptr(), rd.RD_F32,
                              rd.RD_MEM_HOST_ASYNC, rstreams[j])

        def finish(i):     # step i's fields are on the host once its readback stream is done
            pair[i % depth].synchronize(rstreams[i % depth])

        def run(n, t0):      # returns the host time at which each step's fields had arrived
            done = []
            for i in range(n):
                enqueue(i)
                if i >= depth - 1:
                    finish(i - depth + 1)
                    done.append(time.perf_counter() - t0)
            for i in range(max(0, n - depth + 1), n):
                finish(i)
                done.append(time.perf_counter() - t0)
            return done
        mixed.set_timing(False)
        run(max(depth, args.warmup), time.perf_counter())
        torch.cuda.synchronize()
        barrier()
        gc.collect()
        gc.disable()            # no collector pause between a step's enqueue and the next one's
        with ClockSampler(local_rank) as e2e_clk:
            t = time.perf_counter()
            done = run(args.steps, t)
            torch.cuda.synchronize()
            barrier()
            secs = slowest(time.perf_counter() - t)
        gc.enable()
        for dd in pair[1:]:
            dd.close()
        e2e = {"value": deposits * world * args.steps / secs, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * secs / args.steps,
               "step_done_ms": [round(1e3 * v, 2) for v in done],
               "clocks": e2e_clk.summary(),
               "pipeline": f"{depth} detectors on {depth} CUDA streams, readbacks on high-priority streams: "
                           "copies of one step overlap the next step's deposit",
               "host_link": host_link_gbs(Ehs[0], xh)}
    mixed.close()

    # ---------------- FP64 CPU oracle on a bounded sample (rank 0, N = 1 only) ----------------
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs, n_cells, threads, sel, Eo, Bo = oracle_rate(tr, det, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{n_cells} random cells x all {tr.n_part} particles x {tr.n_steps} steps "
                         f"({tr.n_part * tr.n_steps * n_cells:.3g} deposits, {secs:.1f} s)"}
        parity = {"cells": int(n_cells),
                  "mixed_rel_l2_E": float(np.linalg.norm(E_mixed[sel] - Eo) / np.linalg.norm(Eo)),
                  "mixed_rel_l2_B": float(np.linalg.norm(B_mixed[sel] - Bo) / np.linalg.norm(Bo))}

    # measured FMA throughput of this GPU (after the timed regions): a second denominator beside the
    # derived FP32 peak, and the FP64 one for the plain path
    fma32, fma64 = rd.rd_measure_fma_peaks()
    if fp64_info is not None:
        fp64_info["peak_measured_fma_tflops"] = fma64
        fp64_info["frac_of_measured"] = fp64_info["achieved_fp64_tflops"] / fma64 if fma64 > 0 else None

    crossings = st.n_bin_crossings            # of the last timed step (each step starts from zero)
    flops_step = FLOPS_PER_DEPOSIT_MIXED * deposits + FLOPS_PER_CROSSING_MIXED * crossings
    achieved = flops_step / (kernel_ms / 1e3) / 1e12
    peak32, peak_kind = fp32_peak(clocks.get("sm_mhz"))
    traffic = profile_traffic() if tr.n_part == 1000 else None     # the summary covers the full-size launch
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "precision": "mixed: FP32 fields and accumulation, arrival times FP64-anchored at both ends of each step chunk (up to 2048 intervals)",
        "shape": mixed_shape,
        "config": {"workload": undulator_workload(tr.n_part),
                   "deposits_per_step_per_gpu": deposits, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (x,u 192 MB; records 256 MB; fields 1.07 GB)"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "k_deposit_mixed", "achieved": achieved,
                     "peak": peak32, "unit": "TFLOP/s", "frac": achieved / peak32,
                     "peak_kind": peak_kind,
                     "peak_measured_fma": fma32, "frac_of_measured_fma": achieved / fma32 if fma32 > 0 else None,
                     "kernel_ms": kernel_ms, "flops_per_deposit": FLOPS_PER_DEPOSIT_MIXED,
                     "flops_per_crossing": FLOPS_PER_CROSSING_MIXED, "bin_crossings_per_step": crossings,
                     "traffic": traffic},
        "clocks": clocks,
        "fp64_gpu": fp64_info,
        "farfield": ff_info,
        "variants": variants,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "parity_vs_oracle": parity,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
