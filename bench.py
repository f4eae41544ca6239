"""Benchmark: device-timed 2D hull throughput of the segmented QuickHull on GB300.

Workload: 20,000,000 points uniform in the unit disk (seed 0), one set per GPU,
FP32 predicates with certified bound and exact fallback, quadrilateral initial
split.  A step is one full hull (extreme points, initial split, grid-wide
rounds, block finisher, output assembly) through the C ABI with the input
resident in device memory.  L2 is flushed (256 MiB write) before every step;
each step is timed with CUDA events on the launch stream.

Also reported on the same line: the end-to-end figure through qh_hull2d_host
(host input, copies inside the timed region), the roofline of the dominant
kernel (grid-wide rounds, HBM-bound) against the measured copy peak, the CPU
oracle on a bounded sample, the plain-FP64 form and the batched form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank hulls its own copy of the workload (replicas; the
method needs no exchange for independent sets); value = all ranks' points per
second with the max-over-ranks step time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D hull Mpts/s (device-timed) and HBM GB/s vs 8 TB/s; filtered+batched vs plain FP64"
WORKLOAD = "disk-20M: 20,000,000 points i.i.d. uniform in the unit disk (r = sqrt(U), angle = 2 pi U), seed 0"
N_POINTS = 20_000_000


def _set_points(n: int) -> None:
    """Run the disk workload at n points (the benchmark line names the size)."""
    global N_POINTS, WORKLOAD
    if n != N_POINTS:
        N_POINTS = int(n)
        WORKLOAD = (f"disk-{n}: {n:,} points i.i.d. uniform in the unit disk (r = sqrt(U), angle = 2 pi U), "
                    "seed 0 (profiling size, not the benchmark workload)")
CPU_SAMPLE = 10_000_000


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.rows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = self.rows
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[0] or r[0] in self.uuid]
            if mine:
                rows = mine
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce_max(x: float, ws: int, device) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def run_reference(args, ws, rank):
    """The reference arm: the CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth

    pts = synth.disk(N_POINTS, seed=0)
    sample = pts[:2_000_000]
    oracle.build()
    for _ in range(args.warmup):
        oracle.hull2d(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.hull2d(sample)
    dt = (time.perf_counter() - t0) / args.steps
    value = len(sample) / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "first 2,000,000 points of the workload per step"},
        "cpu_baseline": {"value": value, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                         "sample": "monotone-chain oracle, first 2,000,000 points of the workload per step"},
        "e2e": {"value": value, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    _ = np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, batched and CPU-baseline legs")
    ap.add_argument("--points", type=int, default=N_POINTS,
                    help="points of the disk workload (default: the 20M-point benchmark; smaller sizes for profiling)")
    args = ap.parse_args()
    _set_points(args.points)
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import numpy as np
    import torch

    import __graft_entry__ as entry
    import synth

    entry.build()
    import paper_1501_04706_gb300 as qh

    qh.load()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)

    pts = synth.disk(N_POINTS, seed=0)
    d_pts = torch.from_numpy(pts).to(device)
    plan = qh.Plan(N_POINTS, 1)
    out = torch.empty(N_POINTS, dtype=torch.int32, device=device)
    cnt = torch.empty(1, dtype=torch.int32, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream(device)

    def step():
        qh.hull2d(d_pts, plan, out=out, count=cnt, sync=False)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(device)
    h = int(cnt.item())

    # ---------------- device-timed value ----------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(device)
    uuid = str(getattr(props, "uuid", "") or "")
    _barrier(ws)
    torch.cuda.synchronize(device)
    with ClockSampler(uuid) as clocks:
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize(device)
    _barrier(ws)
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    ms_max = _reduce_max(ms, ws, device)
    value = ws * N_POINTS / (ms_max * 1e-3) / 1e6

    # ---------------- roofline of the grid-wide kernel ----------------
    plan.set_tuning(4096, timing=True)
    phase = []
    for _ in range(5):
        flush.fill_(1)
        step()
        st = plan.stats()
        phase.append(st["phase_ms"])
    plan.set_tuning(4096, timing=False)
    rounds_ms = statistics.median(p[0] for p in phase)
    alg_bytes = 16 * st["grid_points"] + 12 * (st["grid_read"] + st["grid_written"])
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (rounds_ms * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "rounds_kernel_disk20M_traffic.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as f:
                tj = json.load(f)
            if tj.get("kernel_rev") == _kernel_rev():
                traffic = tj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "rounds_kernel (extreme points, initial split, grid-wide rounds)",
                "peak_kind": f"{peak_kind} copy bandwidth", "kernel_ms": rounds_ms, "algorithmic_bytes": alg_bytes,
                "phase_ms": {"grid_rounds": rounds_ms, "finisher": statistics.median(p[1] for p in phase),
                             "emit": statistics.median(p[2] for p in phase),
                             "copy": statistics.median(p[3] for p in phase)}}
    whole_gbs = (alg_bytes + 12 * st["small_points"] + 4 * h) / (ms * 1e-3) / 1e9

    # ---------------- end to end through the host-buffer entry point ----------------
    host = torch.from_numpy(pts).pin_memory().numpy()
    host_out = torch.empty(N_POINTS, dtype=torch.int32).pin_memory().numpy()
    for _ in range(2):
        qh.hull2d_host(host, plan, host_out)
    t0 = time.perf_counter()
    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(e2e_steps):
        res = qh.hull2d_host(host, plan, host_out)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = _reduce_max(e2e_s, ws, device)
    e2e = {"value": ws * N_POINTS / e2e_s / 1e6, "unit": "Mpts/s", "h2d_bytes_per_step": 8 * N_POINTS,
           "d2h_bytes_per_step": 4 + 4 * len(res), "ms_per_step": e2e_s * 1e3}

    extras = {}
    cpu = None
    parity = None
    if rank == 0 and not args.no_extras:
        # parity of the benchmarked output, against the oracle (outside any timed region)
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        want = oracle.hull2d(pts[:CPU_SAMPLE])
        cpu_s = time.perf_counter() - t0
        cpu = {"value": CPU_SAMPLE / cpu_s / 1e6, "unit": "Mpts/s", "cores": 1, "kind": "oracle",
               "sample": f"monotone-chain oracle on the first {CPU_SAMPLE:,} points of the workload, one pass"}
        full = oracle.hull2d(pts)
        parity = bool(np.array_equal(out[:h].cpu().numpy(), full))
        _ = want
        # plain FP64 form, same workload
        plan64 = qh.Plan(N_POINTS, 1, prec=qh.PREC_F64)
        for _ in range(3):
            qh.hull2d(d_pts, plan64, out=out, count=cnt, sync=False)
        e64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in e64:
            flush.fill_(1)
            a.record(stream)
            qh.hull2d(d_pts, plan64, out=out, count=cnt, sync=False)
            b.record(stream)
        torch.cuda.synchronize(device)
        ms64 = sum(a.elapsed_time(b) for a, b in e64) / len(e64)
        parity64 = bool(np.array_equal(out[: int(cnt.item())].cpu().numpy(), full))
        extras["fp64_plain"] = {"value": N_POINTS / (ms64 * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms64,
                                "parity": parity64}
        plan64.close()
        # batched form: 4096 sets, one call
        bp, boff = synth.batched()
        d_bp = torch.from_numpy(bp).to(device)
        d_off = torch.from_numpy(boff).to(device)
        planb = qh.Plan(len(bp), len(boff) - 1)
        bo = torch.empty(len(bp), dtype=torch.int32, device=device)
        bc = torch.empty(len(boff) - 1, dtype=torch.int32, device=device)
        for _ in range(3):
            qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
        eb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in eb:
            flush.fill_(1)
            a.record(stream)
            qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
            b.record(stream)
        torch.cuda.synchronize(device)
        msb = sum(a.elapsed_time(b) for a, b in eb) / len(eb)
        extras["batched"] = {"value": len(bp) / (msb * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_step": msb,
                             "sets": len(boff) - 1, "points": int(len(bp))}
        planb.close()

    clk = clocks.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_POINTS, "mode": "quadrilateral initial split",
                   "precision": "f32 filtered predicates + exact fallback", "l2": "flushed before every step",
                   "parallelism": "replicas" if ws > 1 else "single GPU", "hull_vertices": h},
        "gpu_launches": 4 * args.steps,
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
        "whole_path_algorithmic_gbs": whole_gbs, "parity": parity, "extras": extras,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def _kernel_rev() -> str:
    """Content hash of the grid-wide kernel source (ties recorded counters to the code they measured)."""
    import hashlib

    h = hashlib.sha256()
    for f in ("qh_rounds.cu", "qh_internal.cuh", "qh_predicates.cuh"):
        with open(os.path.join(ROOT, "paper_1501_04706_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
