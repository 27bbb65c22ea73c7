#!/usr/bin/env python
"""Throughput benchmark of the quasi-Monte Carlo tracer on one GB300 (or N, weak scaling).

Workload (one step): single scattering of 2^26 packets from a point source in the
flared disk (256^3 FP32 density grid over [-1, 1]^3, HG g = 0.5, albedo 0.6,
p_l = 0.5, observer at 45 degrees), Sobol points, FP32 trace, fixed-point image
accumulation into a 256x256 I/Q/U image, then the reduction to the FP64 image in
units of the source luminosity.  Each step traces the next 2^26 points of the
sequence.  With N ranks every rank traces its own 2^26-packet range per step and the
fixed-point images are summed with one all-reduce before the reduction.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "packets/s and wall time to fixed image RMS error (QMC, learned vs plain), 1 GB300"
PACKETS_PER_STEP = 1 << 26
OPS_PER_CELL = 10          # algorithmic ALU operations per grid-cell visit (see design notes)
SMS, LANES_PER_SM = 152, 128
KERNEL_SOURCES = ["paper_2406_15632_gb300/csrc/qmcrt_device.cuh", "paper_2406_15632_gb300/csrc/qmcrt_trace_single.cu"]
PROFILE = os.path.join(ROOT, "profiles", "trace_single_flared_disk_256.md")
COUNTS = os.path.join(ROOT, "tests", "golden", "workload_counts.json")


def workload_problem():
    from paper_2406_15632_gb300 import scenes as S

    return S.flared_disk_problem(n=256)


def workload_config(n_packets):
    return {"workload": "flared_disk_single_scattering", "grid": "256^3 fp32", "image": "256x256 I/Q/U",
            "packets_per_step_per_gpu": n_packets, "points": "sobol (Joe-Kuo), consecutive index ranges",
            "trace_precision": "fp32 (compensated optical depth)", "accumulate": "int64 fixed point",
            "l2": "flushed between steps (256 MiB write)", "source": "point", "albedo": 0.6, "g": 0.5, "p_l": 0.5,
            "theta_obs_deg": 45}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the trace kernel from the committed ncu summary, if it
    was taken on the current kernel source."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bytes.group(1))


def cells_per_packet():
    with open(COUNTS) as f:
        return json.load(f)["flared_disk_single_scattering"]["cells_per_packet"]


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device, self.proc, self.lines = device, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_cpu_baseline(target_seconds: float = 12.0):
    """The oracle as it stands, on the host cores, on a bounded prefix of the workload."""
    from oracle import oracle as O

    prob = workload_problem()
    threads = O.default_threads()
    n = 1 << 14
    for _ in range(2):  # calibrate on growing samples (thread start-up dominates tiny ones)
        t = time.perf_counter()
        O.trace_single(prob, 1, n, nthreads=threads)
        rate = n / (time.perf_counter() - t)
        n = int(min(max(rate * (target_seconds if _ else 1.5), 1 << 14), 1 << 27))
    t = time.perf_counter()
    O.trace_single(prob, 1, n, nthreads=threads)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "packets/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n} packets of the workload (same Sobol points), FP64 C oracle, {threads} threads, "
                      f"{dt:.1f} s"}


def run_batched():
    """Batched workload: 256 instances (32 inclinations x 8 wavelengths, budgets
    2^floor(U(18, 24))) of the flared disk lit by a finite limb-darkened star, 256x256
    I/Q/U each, FP32.  One graph-captured persistent launch (autotuned decomposition)
    against one regular launch per instance; both produce identical images."""
    import torch

    from paper_2406_15632_gb300 import autotune
    from paper_2406_15632_gb300 import qmcrt as Q
    from paper_2406_15632_gb300 import scenes as S

    prob = S.finite_star_disk_problem(n=256)
    inst = S.batched_instances()
    sc = Q.Scene(prob)
    best = autotune.tune_batch(prob, inst, scene=sc)
    cfg = {k: best[k] for k in ("chunk_log2", "block_size", "ctas_per_sm", "packets_per_thread")}
    B = Q.Batch(prob, inst, scene=sc, **cfg)
    t_graph = autotune.time_batch(B, repeats=3)
    ref = B.accum.clone()
    B.run_each()  # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    B.run_each()
    e1.record()
    e1.synchronize()
    t_seq = e0.elapsed_time(e1)
    same = bool(torch.equal(B.accum, ref))
    n = B.packets()
    return {"workload": "flared disk 256^3, finite star R*=0.05 u=0.6 inverse order, 256 instances",
            "packets": n, "graph_ms": t_graph, "sequential_ms": t_seq, "packets_per_s": n / (t_graph / 1e3),
            "sequential_packets_per_s": n / (t_seq / 1e3), "speedup_at_equal_images": t_seq / t_graph,
            "identical_images": same, "config": cfg, "tuned_over": best.get("tried")}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import oracle as O

    prob = workload_problem()
    threads = O.default_threads()
    n0 = 1 << 14
    t = time.perf_counter()
    O.trace_single(prob, 1, n0, nthreads=threads)
    rate0 = n0 / (time.perf_counter() - t)
    budget = 150.0 / max(args.steps + args.warmup, 1)  # whole run within a few minutes
    n = int(min(max(rate0 * min(budget, 10.0), 4096), PACKETS_PER_STEP))
    for s in range(args.warmup):
        O.trace_single(prob, 1 + s * n, n, nthreads=threads)
    t = time.perf_counter()
    for s in range(args.steps):
        O.trace_single(prob, 1 + (args.warmup + s) * n, n, nthreads=threads)
    dt = time.perf_counter() - t
    value = n * args.steps / dt
    sample = f"{n} packets per step of the workload (consecutive Sobol ranges), FP64 C oracle, {threads} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "packets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(n),
            "cpu_baseline": {"value": value, "unit": "packets/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "packets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=int, default=PACKETS_PER_STEP)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and time-to-error sections")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt as Q
    from paper_2406_15632_gb300 import shard

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    Q.load()
    prob = workload_problem()
    n = args.packets
    total_ranges = (1 << 32) // n - 1
    sc = Q.Scene(prob)
    fb = Q.default_frac_bits(prob, n * world)
    buf = sc.accum_buffer("i64")
    img = torch.empty((1, 3, prob.ny, prob.nx), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def step(s, ev=None):
        first = shard.step_range(s, rank, world, n, total_ranges)
        buf.zero_()
        if ev:
            ev[0].record(stream)
        sc.trace(first, n, buf, frac_bits=fb)
        if ev:
            ev[1].record(stream)
        if world > 1:
            shard.allreduce_image(buf)
        sc.reduce(buf, 1.0 / (n * world), frac_bits=fb, out=img)

    for s in range(args.warmup):
        flush.zero_()
        step(s)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.zero_()
            e = evs[s]
            e[2].record(stream)
            step(args.warmup + s, (e[0], e[1]))
            e[3].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = sum(e[2].elapsed_time(e[3]) for e in evs)
    kern_ms = [e[0].elapsed_time(e[1]) for e in evs]
    t_local = torch.tensor([step_ms, sum(kern_ms)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    step_ms, kern_total = t_local.tolist()
    value = n * world * args.steps / (step_ms / 1e3)

    # end to end through the public call with host buffers (pinned), copies included
    host_grid = torch.from_numpy(prob.grid).pin_memory()
    host_out = torch.empty((1, 3, prob.ny, prob.nx), dtype=torch.float64).pin_memory()
    R = Q.HostRenderer(prob, n * world)
    for s in range(args.warmup):
        R(host_grid, shard.step_range(s, rank, world, n, total_ranges), n, host_out)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        R(host_grid, shard.step_range(args.warmup + s, rank, world, n, total_ranges), n, host_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_ms, op=dist.ReduceOp.MAX)
        dist.barrier()
    e2e_value = n * world * args.steps / (e2e_ms.item() / 1e3)

    if rank != 0:
        dist.destroy_process_group()
        return 0
    peaks = measured_peaks()
    clk = clocks.summary()
    max_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_ops = SMS * LANES_PER_SM * max_mhz * 1e6
    cpp = cells_per_packet()
    kern_avg_s = kern_total / args.steps / 1e3
    achieved_ops = n * cpp * OPS_PER_CELL / kern_avg_s
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "packets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(n),
        "roofline": {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": achieved_ops / peak_ops, "traffic": traffic,
                     "kernel": "k_trace_single<float>", "kernel_ms": kern_avg_s * 1e3,
                     "per_unit": f"{OPS_PER_CELL} ops per cell visit x {cpp:.2f} cells per packet",
                     "peak_basis": f"{SMS} SMs x {LANES_PER_SM} lanes x {max_mhz:.0f} MHz (measured max clock)"},
        "e2e": {"value": e2e_value, "unit": "packets/s", "h2d_bytes_per_step": R.input_bytes(),
                "d2h_bytes_per_step": R.output_bytes()},
        "gpu_launches": 2 * args.steps * 1,
        "clocks": clk,
    }
    if world == 1 and not args.no_extras:
        line["batched"] = run_batched()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
