#!/usr/bin/env python
"""Benchmark of the superstep-scheduled sparse lower-triangular solve on GB300.

Default workload: the random lower-triangular factor with n = 1,000,000 rows,
min(i, 6) distinct columns per row drawn from a 20000-row window, N(0,1)
off-diagonals, diagonal 1 + sum |off|, FP64, one right-hand side.  A step is
one solve L x = b (the schedule is analysed once, outside the timed region,
as the paper's schedule is reused across solves).

Prints ONE JSON line (rank 0).  Key fields:
  value      solved nnz/s over all ranks (device time, CUDA events, inputs resident)
  e2e        the same metric through the public API with host buffers: per step a
             pinned-host -> device copy of b, the solve, and a device -> host copy of x
  roofline   HBM bytes of the solve kernel per launch / its mean duration vs the
             measured copy bandwidth (MEASURED_PEAKS.json)
  cpu_baseline  the CPU oracle (sequential FP64 forward substitution) on host cores

--impl reference runs the CPU oracle itself as the reference arm.
Multi-GPU: every rank solves its own replica (a single factor does not shard);
value = all ranks' nnz / max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "solved nnz/s"
UNIT = "nnz/s"
L2_FLUSH_BYTES = 512 << 20          # > 126 MB L2: written between timed steps
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "random_1m_f64": dict(make=W.config_random_1m, dtype="f64", nrhs=1,
                          desc="random lower factor n=1e6, min(i,6) cols in a 20000-row window, "
                               "N(0,1) off-diagonals, diag 1+sum|off|, FP64, 1 RHS"),
    "lap3d_160_f64": dict(make=W.config_3d_160, dtype="f64", nrhs=1,
                          desc="lower triangle of the 7-point Laplacian on 160^3, FP64, 1 RHS"),
    "lap2d_64_f64": dict(make=W.config_small_2d, dtype="f64", nrhs=1,
                         desc="lower triangle of the 5-point Laplacian on 64x64, FP64, 1 RHS"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="random_1m_f64")
    ap.add_argument("--sync", default=None)
    ap.add_argument("--lanes", type=int, default=None)
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--blocks-per-sm", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="bound of the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def profile_traffic(kernel_tag: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it still matches the source."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.txt")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line:
                k, _, v = line.partition(":")
                fields[k.strip()] = v.strip()
    if fields.get("source_sha1") != kernel_source_sha1():
        return None
    try:
        return float(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_source_sha1():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2503_05408_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:12]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.strip().split(", ") for r in self.tmp.read().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(n, nnz, nrhs, val_bytes, idx_bytes=4, x_bytes=None):
    """nnz*(val+idx) + n*(rowptr + b + x) per right-hand side (matrix read once for the tile)."""
    x_bytes = x_bytes or val_bytes
    return nnz * (val_bytes + idx_bytes) + n * 4 + nrhs * n * 2 * x_bytes


# ------------------------------------------------------------------ CPU baseline
def cpu_oracle_leg(A, b, seconds: float, max_solves: int | None = None):
    """Time the CPU oracle (1 host core, sequential FP64) on whole solves of the factor."""
    import oracle
    x = oracle.solve(A, b)                       # warm (page-in, compile)
    times = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        x = oracle.solve(A, b)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or (max_solves and len(times) >= max_solves):
            break
    per = statistics.median(times)
    nrhs = b.shape[1] if b.ndim == 2 else 1
    return {"value": A.nnz * nrhs / per, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} whole solves of the factor (median {per * 1e3:.2f} ms), 1 thread"}, x, per


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    spec = WORKLOADS[args.workload]
    A, xs, b = spec["make"]()
    import oracle
    oracle.solve(A, b)
    times = []
    for _ in range(args.warmup):
        oracle.solve(A, b)
    budget_end = time.perf_counter() + 120.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve(A, b)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > budget_end:
            break
    total = sum(times)
    value = A.nnz * spec["nrhs"] * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": spec["dtype"],
            "data": "synthetic",
            "config": {"workload": args.workload, "description": spec["desc"], "n": A.n, "nnz": A.nnz,
                       "nrhs": spec["nrhs"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1,
                             "sample": f"{len(times)} whole sequential FP64 solves on 1 host thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    import paper_2503_05408_gb300 as sp

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    spec = WORKLOADS[args.workload]
    A, xs, b_np = spec["make"]()
    nrhs = spec["nrhs"]
    t0 = time.perf_counter()
    plan = sp.Plan(A, mode="levels", device=local)
    analyze_s = time.perf_counter() - t0
    st = plan.stats()

    tdtype = torch.float64
    b = torch.from_numpy(np.ascontiguousarray(b_np[:, 0])).to(f"cuda:{local}", tdtype)
    x = torch.empty_like(b)
    opts = dict(sync=args.sync, lanes=args.lanes, threads=args.threads, blocks_per_sm=args.blocks_per_sm)
    opts = {k: v for k, v in opts.items() if v is not None}
    if "sync" not in opts:
        opts.update(plan.autotune(b, x))
    _, rep = plan.solve(b, x, **opts)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()

    def step():
        plan.solve(b, x, report=False, **opts)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for e0, e1 in ev:
        flush.zero_()                              # L2 flushed between timed steps
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    durs = [e0.elapsed_time(e1) * 1e-3 for e0, e1 in ev]
    dev_total = sum(durs)

    # end to end through the public API with host buffers
    b_host = torch.from_numpy(np.ascontiguousarray(b_np[:, 0])).to(tdtype).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    b2 = torch.empty_like(b)
    x2 = torch.empty_like(b)
    for _ in range(args.warmup):
        b2.copy_(b_host, non_blocking=True)
        plan.solve(b2, x2, report=False, **opts)
        x_host.copy_(x2, non_blocking=True)
    torch.cuda.synchronize()
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist:
        dist.barrier()
    for e0, e1 in ev2:
        flush.zero_()
        e0.record(stream)
        b2.copy_(b_host, non_blocking=True)
        plan.solve(b2, x2, report=False, **opts)
        x_host.copy_(x2, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    e2e_total = sum(e0.elapsed_time(e1) * 1e-3 for e0, e1 in ev2)
    if dist:
        t = torch.tensor([dev_total, e2e_total], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_total, e2e_total = float(t[0]), float(t[1])

    nnz_step = A.nnz * nrhs
    value = nnz_step * args.steps * world / dev_total
    e2e_value = nnz_step * args.steps * world / e2e_total
    mean_s = dev_total / args.steps
    bytes_launch = algorithmic_bytes(A.n, A.nnz, nrhs, 8)
    peak, peak_src = measured_peaks()
    achieved = bytes_launch / mean_s / 1e9
    kernel_tag = f"solve_{SYNC_TAG.get(rep['sync_name'], rep['sync_name'])}_{args.workload}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": spec["dtype"],
        "data": "synthetic (seeded generator, see config.description)",
        "config": {"workload": args.workload, "description": spec["desc"], "n": A.n, "nnz": A.nnz,
                   "nrhs": nrhs, "parallelism": f"replicas x{world}", "l2": "flushed between steps",
                   "levels": st["levels"], "supersteps": st["supersteps"], "schedule": "levels",
                   "sync": rep["sync_name"], "lanes": rep["lanes"], "grid": rep["grid"],
                   "threads": rep["threads"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profile_traffic(kernel_tag),
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                     else "fallback 6.8 TB/s", "kernel": kernel_tag,
                     "algorithmic_bytes_per_launch": bytes_launch},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(b_host.numel() * 8),
                "d2h_bytes_per_step": int(x_host.numel() * 8)},
        "gpu_launches": args.steps,
        "clocks": clk,
        "sync_points_per_step": rep["barriers"] + rep["flag_waits"],
        "analyze_ms": analyze_s * 1e3,
    }
    if rank == 0 and not args.no_cpu_baseline:
        cpu, x_or, cpu_s = cpu_oracle_leg(A, b_np, args.cpu_seconds)
        line["cpu_baseline"] = cpu
        import oracle
        line["err_vs_oracle"] = oracle.rel_error(x.double().cpu().numpy(), x_or)
        gain = cpu_s - mean_s
        line["amortization"] = (analyze_s / gain) if gain > 0 else None   # Eq. 7.1
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


SYNC_TAG = {"grid": "grid", "flags": "flags", "cta": "cta"}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
