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
    """The reference arm: the CPU oracle on the whole workload, timed on all host cores (the oracle's
    monotone chain on contiguous chunks in threads, then on the union of the chunk hulls; same output)."""
    if rank != 0:
        return
    import oracle
    import synth

    pts = synth.disk(N_POINTS, seed=0)
    oracle.build_parallel()
    cores = oracle.host_threads()
    for _ in range(args.warmup):
        oracle.hull2d_parallel(pts, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.hull2d_parallel(pts, cores)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = len(pts) / dt / 1e6
    sample = (f"whole workload ({len(pts):,} points) per step: the oracle's monotone chain with exact predicates "
              f"on {cores} contiguous chunks in {cores} threads, then on the union of the chunk hulls")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "Mpts/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, batched and CPU-baseline legs")
    ap.add_argument("--study", choices=["modes", "sweep", "profile", "configs", "sorted"], default=None,
                    help="instead of the benchmark line: the five workloads in their stated forms (configs), "
                         "quadrilateral vs chord initial split (modes), "
                         "uniform-square size sweep (sweep), per-sub-procedure times (profile) or the x-sorted "
                         "form of the rounds against the unsorted one (sorted), one JSON line each")
    ap.add_argument("--cases", default=None,
                    help="sorted study: comma-separated workloads (disk-20M, circle-20M, degenerate-16M, "
                         "square-100K, square-2M, square-20M; default all)")
    ap.add_argument("--points", type=int, default=N_POINTS,
                    help="points of the disk workload (default: the 20M-point benchmark; smaller sizes for profiling)")
    args = ap.parse_args()
    _set_points(args.points)
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.study:
        return run_study(args.study, args.cases)

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
    # qh_hull2d_host reads back the count with the first min(n, 65536) indices, then any indices beyond
    eager = min(N_POINTS, 65536)
    e2e = {"value": ws * N_POINTS / e2e_s / 1e6, "unit": "Mpts/s", "h2d_bytes_per_step": 8 * N_POINTS,
           "d2h_bytes_per_step": 4 + 4 * eager + 4 * max(0, len(res) - eager), "ms_per_step": e2e_s * 1e3}

    extras = {}
    cpu = None
    parity = None
    if rank == 0 and not args.no_extras:
        # parity of the benchmarked output, against the oracle (outside any timed region)
        import oracle

        oracle.build()
        oracle.build_parallel()
        cores = oracle.host_threads()
        t0 = time.perf_counter()
        full = oracle.hull2d(pts)
        cpu1_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        full_par = oracle.hull2d_parallel(pts, cores)
        cpun_s = time.perf_counter() - t0
        cpu = {"value": N_POINTS / cpun_s / 1e6, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
               "sample": (f"the whole workload ({N_POINTS:,} points), one pass: the oracle's monotone chain on "
                          f"{cores} contiguous chunks in {cores} threads, then on the union of the chunk hulls"),
               "same_output_as_single_thread": bool(np.array_equal(full_par, full)),
               "single_thread": {"value": N_POINTS / cpu1_s / 1e6, "unit": "Mpts/s", "cores": 1,
                                 "sample": f"the whole workload ({N_POINTS:,} points), one pass"}}
        parity = bool(np.array_equal(out[:h].cpu().numpy(), full))
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
        tuned = planb.autotune(d_bp, d_off, out=bo, counts=bc, reps=2)  # block size, CTAs per SM, cutover
        for _ in range(3):
            qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
        # one CUDA-graph-captured launch sequence for the whole batch
        launch = "cuda graph"
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
            replay = graph.replay
        except Exception as exc:  # capture refused: time the eager launches and say so
            launch = f"eager (graph capture failed: {type(exc).__name__})"
            torch.cuda.synchronize(device)
            replay = lambda: qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
        replay()
        torch.cuda.synchronize(device)
        eb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in eb:
            flush.fill_(1)
            a.record(stream)
            replay()
            b.record(stream)
        torch.cuda.synchronize(device)
        msb = sum(a.elapsed_time(b) for a, b in eb) / len(eb)
        # whole-path algorithmic bytes of the batch: the grid kernel's (16 B per point of the sets it tiles,
        # 12 B per live point its rounds read or write), 12 B per point the block finisher reads (whole small
        # sets and small segments), 4 B per output index
        stb = planb.stats()
        hb = int(bc.sum().item())
        alg_b = (16 * stb["grid_points"] + 12 * (stb["grid_read"] + stb["grid_written"]) + 12 * stb["small_points"]
                 + 4 * hb)
        gbs_b = alg_b / (msb * 1e-3) / 1e9
        peak_b, peak_kind_b = _peaks()
        # the same sets, one plain-FP64 call per set on one stream
        nsets = len(boff) - 1
        plan1 = qh.Plan(int(np.max(np.diff(boff))), 1, prec=qh.PREC_F64)
        po = torch.empty(len(bp), dtype=torch.int32, device=device)
        pc = torch.empty(nsets, dtype=torch.int32, device=device)

        def per_instance():
            for i in range(nsets):
                a0, a1 = int(boff[i]), int(boff[i + 1])
                qh.hull2d(d_bp[a0:a1], plan1, out=po[a0:a1], count=pc[i:i + 1], sync=False)

        per_instance()
        torch.cuda.synchronize(device)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        a.record(stream)
        per_instance()
        b.record(stream)
        torch.cuda.synchronize(device)
        msi = a.elapsed_time(b)
        cb, cp = bc.cpu().numpy(), pc.cpu().numpy()
        ob, op = bo.cpu().numpy(), po.cpu().numpy()
        same = bool(np.array_equal(cb, cp)) and all(
            np.array_equal(ob[boff[i]:boff[i] + cb[i]], op[boff[i]:boff[i] + cp[i]]) for i in range(nsets))
        extras["batched"] = {"value": len(bp) / (msb * 1e-3) / 1e6, "unit": "Mpts/s", "ms_per_step": msb,
                             "sets": nsets, "points": int(len(bp)), "launch": launch, "autotuned": tuned,
                             "per_instance_fp64": {"value": len(bp) / (msi * 1e-3) / 1e6, "unit": "Mpts/s",
                                                   "ms": msi, "calls": nsets, "same_hulls_as_batched": same},
                             "speedup_vs_per_instance_fp64": msi / msb,
                             "roofline": {"bound": "hbm", "achieved": gbs_b, "peak": peak_b, "unit": "GB/s",
                                          "frac": gbs_b / peak_b, "algorithmic_bytes": alg_b,
                                          "peak_kind": f"{peak_kind_b} copy bandwidth",
                                          "scope": "whole batched call (grid kernel, finisher, emit, copy)"}}
        plan1.close()
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


# Unit-square times of the paper's GPU pipeline on a Tesla K20c (Table 2), ms: (Mode 1, Mode 2).
PAPER_SQUARE_MS = {100_000: (37.2, 61.7), 200_000: (36.4, 65.7), 500_000: (41.7, 69.2), 1_000_000: (44.8, 73.9),
                   2_000_000: (55.9, 86.2), 5_000_000: (77.9, 118.5), 10_000_000: (124.7, 161.7),
                   20_000_000: (206.0, 272.5)}


def _time_hull(qh, torch, d_pts, plan, flush, reps: int = 5):
    """Median device time (ms) of one hull with the L2 flushed before each, and the plan's stats."""
    stream = torch.cuda.current_stream()
    out = torch.empty(max(d_pts.shape[0], 1), dtype=torch.int32, device=d_pts.device)
    cnt = torch.empty(1, dtype=torch.int32, device=d_pts.device)
    for _ in range(2):
        qh.hull2d(d_pts, plan, out=out, count=cnt, sync=False)
    times = []
    for _ in range(reps):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qh.hull2d(d_pts, plan, out=out, count=cnt, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2], plan.stats(), int(cnt.item())


def run_study(study: str, cases: str | None = None) -> None:
    """Studies beside the benchmark (one JSON line per case):
    modes   -- the quadrilateral initial split (the paper's Mode 1) against the chord split (Mode 2) on the
               single-set workloads: device time and live points per generation;
    sweep   -- uniform unit square from 100K to 20M points in both modes, with the paper's K20c times (Table 2)
               as context;
    profile -- the time of each sub-procedure (set prep, extreme points, initial split, every grid round,
               block finisher, output) on every workload, from the device clock and CUDA events;
    sorted  -- the x-sorted form of the rounds (qh_hull2d_sorted, the paper's arrangement) against the
               unsorted plan path on the same input: device times, its phases, identical hulls, and the
               algorithmic bytes of both."""
    import numpy as np
    import torch

    import __graft_entry__ as entry
    import synth

    entry.build()
    import paper_1501_04706_gb300 as qh

    qh.load()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    modes = [("quadrilateral", qh.MODE_QUAD), ("chord", qh.MODE_CHORD)]
    if study == "configs":
        return _study_configs(qh, torch, np, synth, device, flush)
    if study == "sorted":
        return _study_sorted(qh, torch, np, synth, device, flush, cases)
    if study in ("modes", "profile"):
        cases = [("square-100K", synth.square()), ("disk-20M", synth.disk()), ("circle-20M", synth.circle()),
                 ("degenerate-16M", synth.degenerate())]
        for name, pts in cases:
            d_pts = torch.from_numpy(pts).to(device)
            plan = qh.Plan(len(pts), 1)
            for mname, mode in (modes if study == "modes" else modes[:1]):
                plan.set_flags(mode, qh.PREC_F32)
                plan.set_tuning(4096, timing=study == "profile")
                ms, st, h = _time_hull(qh, torch, d_pts, plan, flush)
                line = {"study": study, "workload": name, "mode": mname, "n": len(pts), "hull_vertices": h,
                        "ms": ms, "mpts_per_s": len(pts) / (ms * 1e-3) / 1e6}
                if study == "modes":
                    live = [int(v) for v in st["live"]]
                    while live and live[-1] == 0:
                        live.pop()
                    line.update({"live_per_generation": live, "grid_rounds": st["global_rounds"],
                                 "generations": st["generations"], "exact_orient": st["exact_orient"],
                                 "exact_compare": st["exact_compare"]})
                else:
                    g = [round(v, 1) for v in st["grid_phase_us"] if v > 0]
                    ph = st["phase_ms"]
                    line.update({"us": {"set_prep": g[0] if g else None, "extreme_points": g[1] if len(g) > 1 else None,
                                        "initial_split": g[2] if len(g) > 2 else None, "grid_rounds": g[3:],
                                        "block_finisher": round(ph[1] * 1e3, 1),
                                        "output_emit_copy": round((ph[2] + ph[3]) * 1e3, 1)},
                                 "timing_note": "per-phase events and device-clock stamps on; ms is the timed hull"})
                print(json.dumps(line), flush=True)
            plan.close()
            del d_pts
    else:
        for n in sorted(PAPER_SQUARE_MS):
            pts = synth.square(n)
            d_pts = torch.from_numpy(pts).to(device)
            plan = qh.Plan(n, 1)
            for k, (mname, mode) in enumerate(modes):
                plan.set_flags(mode, qh.PREC_F32)
                ms, st, h = _time_hull(qh, torch, d_pts, plan, flush)
                print(json.dumps({"study": "sweep", "workload": f"square-{n}", "mode": mname, "n": n,
                                  "hull_vertices": h, "ms": ms, "mpts_per_s": n / (ms * 1e-3) / 1e6,
                                  "paper_k20c_ms": PAPER_SQUARE_MS[n][k],
                                  "paper_note": "Table 2, Tesla K20c, timed region unstated: context only"}),
                      flush=True)
            plan.close()
            del d_pts


def _alg_bytes(n: int, live, h: int) -> int:
    """Algorithmic bytes of the path: 8n (extreme points) + 8n (initial split read) + 12 L0 (its writes)
    + sum over later generations of 12 (L_{r-1} + L_r) (read and write) + 4h (output)."""
    live = [int(v) for v in live]
    b = 16 * n + 4 * h + (12 * live[0] if live else 0)
    for r in range(1, len(live)):
        b += 12 * (live[r - 1] + live[r])
    return b


def _alg_bytes_sorted(n: int, live, items: int, h: int) -> dict:
    """Algorithmic bytes of the x-sorted form by step: extreme points 8n; first split 8n read and 8 B
    written per item (x key, payload); radix sort 4 passes of 20 B per item (4 read by the histogram,
    8 read and 8 written by the scatter); gather 4 B payload, 8 B coordinates and 12 B written per item;
    round r: 8 + 8 + 12 B read per point of generation r - 1 (farthest point, count, move) and 12 B written
    per point of generation r; output 8h.  Heads (at most h per round) are not counted."""
    live = [int(v) for v in live]
    rounds = sum(28 * live[r - 1] + 12 * live[r] for r in range(1, len(live)))
    if len(live) > 0:
        rounds += 28 * live[-1]  # the last round reads its generation and keeps no point
    b = {"extreme_points": 8 * n, "first_split": 8 * n + 8 * items, "sort": 80 * items, "gather": 24 * items,
         "rounds": rounds, "output": 8 * h}
    b["total"] = sum(b.values())
    return b


def _study_sorted(qh, torch, np, synth, device, flush, cases):
    """The x-sorted form against the unsorted plan path, both initial splits, same plan and input."""
    all_cases = [("disk-20M", synth.disk), ("circle-20M", synth.circle), ("degenerate-16M", synth.degenerate),
                 ("square-100K", lambda: synth.square(100_000)), ("square-2M", lambda: synth.square(2_000_000)),
                 ("square-20M", lambda: synth.square(20_000_000))]
    want = set(cases.split(",")) if cases else None
    for name, gen in all_cases:
        if want is not None and name not in want:
            continue
        pts = gen()
        n = len(pts)
        d_pts = torch.from_numpy(pts).to(device)
        out = torch.empty(n, dtype=torch.int32, device=device)
        cnt = torch.empty(1, dtype=torch.int32, device=device)
        plan = qh.Plan(n, 1)
        for mname, mode in (("quadrilateral", qh.MODE_QUAD), ("chord", qh.MODE_CHORD)):
            plan.set_flags(mode, qh.PREC_F32)
            ms_u, st_u, h = _time_hull(qh, torch, d_pts, plan, flush)
            ref = qh.hull2d(d_pts, plan).cpu().numpy()
            got = qh.hull2d_sorted(d_pts, plan, out, cnt).cpu().numpy()
            times = []
            for _ in range(5):
                flush.fill_(1)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                qh.hull2d_sorted(d_pts, plan, out, cnt)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            times.sort()
            ms_s = times[len(times) // 2]
            plan.set_tuning(4096, timing=True)
            flush.fill_(1)
            qh.hull2d_sorted(d_pts, plan, out, cnt)
            st_s = plan.stats()
            plan.set_tuning(4096, timing=False)
            live = [int(v) for v in st_s["live"]]
            items = live[0] + (2 if mname == "chord" else 4)  # survivors of the first split and the polygon
            ph = st_s["phase_ms"]
            print(json.dumps({
                "study": "sorted", "workload": name, "mode": mname, "n": n, "hull_vertices": h,
                "ms_unsorted": ms_u, "ms_sorted": ms_s, "sorted_over_unsorted": ms_s / ms_u,
                "same_hull": bool(np.array_equal(got, ref)), "same_live_counts": st_s["live"] == st_u["live"],
                "generations": st_s["generations"],
                "sorted_phases_ms": {"extreme_points_and_first_split": ph[0], "sort_and_gather": ph[1],
                                     "rounds": ph[2], "output": ph[3], "total": ph[4]},
                "algorithmic_gb": {"unsorted": _alg_bytes(n, st_u["live"], h) / 1e9,
                                   "sorted": {k: v / 1e9 for k, v in _alg_bytes_sorted(n, live, items, h).items()}},
                "round_bytes_per_point": {"unsorted": {"read": 12, "written": 12},
                                          "sorted": {"read": 28, "written": 12}},
                "note": "sorted form: one host check of the end flag per 8 rounds, inside the timed region"}),
                flush=True)
        plan.close()
        del d_pts


def _study_configs(qh, torch, np, synth, device, flush):
    """The five workloads in the forms they are stated in: device time, Mpts/s, algorithmic GB/s against
    8 TB/s nominal and the measured copy peak, exact-fallback rates, parity with the oracle."""
    import oracle

    peak, _ = _peaks()
    runs = [("1: square-100K", synth.square, [("plain FP64", qh.PREC_F64)]),
            ("2: disk-20M", synth.disk, [("plain FP64", qh.PREC_F64), ("FP32 filtered", qh.PREC_F32)]),
            ("3: circle-20M", synth.circle, [("FP32 filtered", qh.PREC_F32)]),
            ("4: degenerate-16M", synth.degenerate, [("FP32 filtered", qh.PREC_F32)])]
    for name, gen, forms in runs:
        pts = gen()
        want = oracle.hull2d(pts)
        d_pts = torch.from_numpy(pts).to(device)
        plan = qh.Plan(len(pts), 1)
        for form, prec in forms:
            plan.set_flags(qh.MODE_QUAD, prec)
            ms, st, h = _time_hull(qh, torch, d_pts, plan, flush, reps=9)
            got = qh.hull2d(d_pts, plan).cpu().numpy()
            ab = _alg_bytes(len(pts), st["live"], h)
            gbs = ab / (ms * 1e-3) / 1e9
            print(json.dumps({"study": "configs", "config": name, "form": form, "n": len(pts), "hull_vertices": h,
                              "ms": ms, "mpts_per_s": len(pts) / (ms * 1e-3) / 1e6, "algorithmic_gb": ab / 1e9,
                              "algorithmic_gbs": gbs, "frac_of_8tbs": gbs / 8000.0, "frac_of_measured_copy": gbs / peak,
                              "exact_orient_per_point": st["exact_orient"] / len(pts),
                              "exact_compare": st["exact_compare"], "parity": bool(np.array_equal(got, want))}),
                  flush=True)
        plan.close()
        del d_pts
    bp, boff = synth.batched()
    d_bp = torch.from_numpy(bp).to(device)
    d_off = torch.from_numpy(boff).to(device)
    planb = qh.Plan(len(bp), len(boff) - 1)
    bo = torch.empty(len(bp), dtype=torch.int32, device=device)
    bc = torch.empty(len(boff) - 1, dtype=torch.int32, device=device)
    tuned = planb.autotune(d_bp, d_off, out=bo, counts=bc, reps=2)
    qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        qh.hull2d_batched(d_bp, d_off, planb, out=bo, counts=bc)
    times = []
    for _ in range(9):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    ms = times[len(times) // 2]
    st = planb.stats()
    print(json.dumps({"study": "configs", "config": "5: batched 4096 sets", "form": "FP32 filtered, one CUDA graph",
                      "autotuned": tuned,
                      "n": int(len(bp)), "ms": ms, "mpts_per_s": len(bp) / (ms * 1e-3) / 1e6,
                      "exact_orient_per_point": st["exact_orient"] / len(bp), "exact_compare": st["exact_compare"],
                      "parity": "per set in tests/test_gpu_parity.py (batched == oracle per set)"}), flush=True)
    planb.close()


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
