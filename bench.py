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
OPS_PER_PACKET = 150       # setup and transcendentals of one packet's single scattering (emission,
                           # forced depth, peel-off phase function and Stokes, binning)
SMS, LANES_PER_SM = 152, 128
KERNEL_SOURCES = ["paper_2406_15632_gb300/csrc/qmcrt_device.cuh", "paper_2406_15632_gb300/csrc/qmcrt_trace_single.cu",
                  "paper_2406_15632_gb300/csrc/qmcrt_api.cu"]  # the kernel and the host side of its packet order
PROFILE = os.path.join(ROOT, "profiles", "trace_single_flared_disk_256.md")
COUNTS = os.path.join(ROOT, "tests", "golden", "workload_counts.json")


def workload_problem():
    from paper_2406_15632_gb300 import scenes as S

    return S.flared_disk_problem(n=256)


def workload_config(n_packets):
    """The workload (flared disk of Sec. 5: g 0.5, albedo 0.6, p_l 0.5, observer at 45 deg,
    point source, Sobol points in aligned 2^26 blocks, FP32 trace), in a few keys."""
    return {"workload": "flared_disk_single_scattering", "grid": "256^3 fp32", "image": "256x256 I/Q/U",
            "packets_per_step_per_gpu": n_packets, "accumulate": "int64 fixed point", "l2": "flushed (256 MiB write)"}


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


def cells_per_packet(workload="flared_disk_single_scattering", key="cells_per_packet"):
    with open(COUNTS) as f:
        return json.load(f)[workload][key]


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
    # one core, as the paper times its own code (a shorter prefix of the same points)
    n1 = max(1 << 12, int(n / threads / 4))
    t = time.perf_counter()
    O.trace_single(prob, 1, n1, nthreads=1)
    dt1 = time.perf_counter() - t
    return {"value": n / dt, "unit": "packets/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n} packets of the workload (same Sobol points), FP64 C oracle, {threads} threads, "
                      f"{dt:.1f} s",
            "sample_short": f"first {n} packets, {threads} threads",
            "single_core": {"value": n1 / dt1, "unit": "packets/s", "sample": f"first {n1} packets, 1 thread, "
                                                                              f"{dt1:.1f} s"}}


def run_multiple_scattering(log2_n=24, repeats=3):
    """Clumpy envelope (128^3, 20 orders, forced, roulette 1e-4, 512x512 I/Q/U), 2^24
    Sobol packets per run, FP32 trace, int64 accumulation: packets/s over `repeats`
    timed runs after one warm-up, and its ALU roofline fraction with the oracle's count
    of cells visited per packet."""
    import torch

    from paper_2406_15632_gb300 import qmcrt as Q
    from paper_2406_15632_gb300 import scenes as S

    prob = S.clumpy_problem(n=128)
    sc = Q.Scene(prob)
    n = 1 << log2_n
    fb = Q.default_frac_bits(prob, n)
    buf = sc.accum_buffer("i64")
    stream = torch.cuda.current_stream()

    def run(k):
        buf.zero_()
        sc.trace(n * (k + 1), n, buf, frac_bits=fb)
    run(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(repeats):
        run(k + 1)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / repeats
    ref = buf.clone()
    # the same packets order by order, live packets regrouped between orders
    ws = sc.wavefront_workspace(n)

    def run_wave(k):
        buf.zero_()
        sc.trace_wavefront(n * (k + 1), n, buf, ws, frac_bits=fb)
    run_wave(0)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(repeats):
        run_wave(k + 1)
    e1.record(stream)
    e1.synchronize()
    ms_wave = e0.elapsed_time(e1) / repeats
    same = bool(torch.equal(buf, ref))
    cpp = cells_per_packet("clumpy_multiple_scattering", key="cells_per_packet_single_pass")
    peak = SMS * LANES_PER_SM * measured_peaks().get("sm_max_mhz", 2070.0) * 1e6
    per_unit = (f"{OPS_PER_CELL} ops per cell visit x {cpp:.1f} cells per packet (oracle count, without the "
                f"forced steps' second passes)")

    def roofline(t_ms, kernel):
        ops = n * cpp * OPS_PER_CELL / (t_ms / 1e3)
        return {"bound": "alu", "achieved": ops / 1e12, "peak": peak / 1e12, "unit": "Tops/s", "frac": ops / peak,
                "kernel": kernel, "per_unit": per_unit}
    # the library's faster path for this workload (the wavefront) first; the one-kernel
    # tracer beside it, with identical images
    return {"workload": "clumpy envelope 128^3, point source, 20 orders, forced, roulette 1e-4, 512x512 I/Q/U, "
                        "FP32 trace, int64 accumulate", "packets": n, "path": "wavefront",
            "ms": ms_wave, "packets_per_s": n / (ms_wave / 1e3),
            "roofline": roofline(ms_wave, "k_wave_order<float> + k_wave_first<float> (+ sort)"),
            "one_kernel": {"ms": ms, "packets_per_s": n / (ms / 1e3), "identical_images": same,
                           "roofline": roofline(ms, "k_trace_multiple<float>")}}


def run_observers(n_obs=8, log2_n=24):
    """One trace of the 256^3 disk feeding n_obs observers (inclinations 0..90 degrees)
    against n_obs single-observer traces of the same packets; the stacks are identical
    (checked), so the speedup is at equal images."""
    import torch

    from paper_2406_15632_gb300 import qmcrt as Q

    prob = workload_problem()
    sc = Q.Scene(prob)
    n = 1 << log2_n
    fb = Q.default_frac_bits(prob, n)
    angles = [(math.radians(90.0 * k / (n_obs - 1)), 0.0) for k in range(n_obs)]
    stack = torch.zeros((n_obs, 1, 3, prob.ny, prob.nx), dtype=torch.int64, device="cuda")
    sep = torch.zeros_like(stack)
    scenes = [Q.Scene(prob.replace(theta_obs=th, phi_obs=ph), grid_device=sc.grid) for th, ph in angles]

    def together():
        stack.zero_()
        sc.trace_observers(angles, n, n, stack, frac_bits=fb)

    def apart():
        sep.zero_()
        for o, s_o in enumerate(scenes):
            s_o.trace(n, n, sep[o], frac_bits=fb)
    together()
    apart()
    _, ms_together = _timed(together)
    _, ms_apart = _timed(apart)
    return {"workload": f"flared disk 256^3 single scattering, {n_obs} observers at inclinations 0-90 deg, "
                        "256x256 I/Q/U each, FP32 trace, int64 accumulate",
            "packets": n, "observers": n_obs, "one_trace_ms": ms_together, "separate_traces_ms": ms_apart,
            "packet_observers_per_s": n * n_obs / (ms_together / 1e3), "speedup": ms_apart / ms_together,
            "identical_images": bool(torch.equal(stack, sep))}


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
    # time to error: both forms give the same image per instance, so at each instance's
    # budget they reach the same error; that error is estimated per instance from two
    # independently Owen-scrambled batches (the replicate spread, no reference)
    reps = []
    for seed in (1, 2):
        R = Q.Batch(prob.replace(generator="sobol_owen", seed=seed), inst, scene=sc, **cfg)
        R.run()
        torch.cuda.synchronize()
        reps.append(R.out[:, 0].clone())
        del R
    per = [_replicate_error([reps[0][i], reps[1][i]]) for i in range(len(inst))]
    return {"workload": "flared disk 256^3, finite star R*=0.05 u=0.6 inverse order, 256 instances",
            "packets": n, "graph_ms": t_graph, "sequential_ms": t_seq, "packets_per_s": n / (t_graph / 1e3),
            "sequential_packets_per_s": n / (t_seq / 1e3), "speedup_at_equal_images": t_seq / t_graph,
            "identical_images": same, "config": cfg, "tuned_over": best.get("tried"),
            "time_to_error": {"per_instance_rms_median": statistics.median(per), "per_instance_rms_max": max(per),
                              "error": "RMS relative of each instance's I image from two Owen-scrambled batches",
                              "batched_ms": t_graph, "separate_ms": t_seq, "speedup": t_seq / t_graph}}


def _timed(fn):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def _norms(img, ref):
    """(RMS relative = ||A - B||_2 / ||B||_2, L1 relative = sum |A - B| / sum |B|) of the I images."""
    d = img - ref
    return float(d.norm() / ref.norm()), float(d.abs().sum() / ref.abs().sum())


def _time_at(points, target):
    """Wall time at which an arm reaches `target` error: log-log interpolation between
    the ladder points (time, error) that bracket it, else extrapolation along the last
    two points (flagged)."""
    pts = sorted(points)
    for (t0, e0), (t1, e1) in zip(pts, pts[1:]):
        if e0 >= target >= e1 and e0 > e1:
            f = math.log(e0 / target) / math.log(e0 / e1)
            return math.exp(math.log(t0) + f * math.log(t1 / t0)), False
    (t0, e0), (t1, e1) = pts[-2], pts[-1]
    if e1 >= e0:
        return None, True
    slope = math.log(t1 / t0) / math.log(e0 / e1)
    return t1 * (e1 / target) ** slope, True


def _reference_image(Q, prob, grid, render_log2, seeds, accum):
    """Converged reference: mean of Owen-scrambled Sobol images with independent seeds,
    and the estimated RMS error of that mean (sample variance across seeds / seeds)."""
    import torch

    imgs = []
    for seed in seeds:
        sc = Q.Scene(prob.replace(generator="sobol_owen", seed=seed), grid_device=grid)
        n = 1 << render_log2
        fb = Q.default_frac_bits(sc.prob, n) if accum == "i64" else 0
        buf = sc.accum_buffer(accum)
        sc.trace(n, n, buf, accum=accum, frac_bits=fb)  # points n .. 2n - 1: one whole net block
        imgs.append(sc.reduce(buf, 1.0 / n, accum=accum, frac_bits=fb)[0, 0].clone())
    stack = torch.stack(imgs)
    ref = stack.mean(0)
    var_of_mean = stack.var(0, unbiased=True).sum() / len(seeds)
    return ref, float(var_of_mean.sqrt() / ref.norm()), len(seeds) << render_log2


def _ladder(render, ladder, ref, ref_err):
    rows = []
    for lg in ladder:
        img, ms = render(1 << lg)
        rms, l1 = _norms(img, ref)
        corr = math.sqrt(max(rms * rms - ref_err * ref_err, 0.0))
        rows.append({"log2_n": lg, "ms": ms, "rms": rms, "rms_minus_reference": corr, "l1": l1})
    return rows


def _tte_summary(arms, targets, overhead_ms=None, key="rms_minus_reference"):
    """Per target error and arm: render time at that error (log-log interpolation on the
    ladder, or extrapolation along its last two points, flagged) plus the arm's fixed
    overhead (training), in ms.  key: the ladder rows' error column."""
    overhead_ms = overhead_ms or {}
    out = {}
    for tgt in targets:
        row = {}
        for name, rows in arms.items():
            pts = [(r["ms"], r[key]) for r in rows if r[key] > 0]
            t, extrap = _time_at(pts, tgt) if len(pts) >= 2 else (None, True)
            row[name] = {"ms": None if t is None else t + overhead_ms.get(name, 0.0), "extrapolated": extrap}
        out[f"{tgt:g}"] = row
    return out


SOBOL_BLOCK_LOG2 = 31  # a Sobol point set has 2^32 points: renders above 2^31 packets use several scrambles


def _replicate_error(imgs):
    """RMS relative error of one render, estimated from R independent randomized renders
    (Owen scrambles or PRNG seeds): sqrt(sum_r ||A_r - mean||^2 / (R - 1)) / ||mean||, no
    reference image needed (the replicates' mean is unbiased, their spread the error)."""
    import torch

    stack = torch.stack(imgs)
    mean = stack.mean(0)
    var = ((stack - mean) ** 2).sum() / (len(imgs) - 1)
    return float(var.sqrt() / mean.norm())


def run_time_to_error_learned(ladder=(20, 22, 24, 26, 28), mc_ladder=None, replicates=2, n_log_log2=20, epochs=2,
                              batch_log2=16, lr=2e-2, mix=0.1, weight="l2", targets=(0.05, 0.03, 1e-2, 1e-3),
                              chunk_log2=22):
    """Clumpy envelope (128^3, total radial tau 5, 20 orders, roulette at 1e-4, 512x512
    I/Q/U): wall time to a fixed RMS error of the I image for plain QMC, the learned
    proposal (warp trained on the tracer's own log of 2^n_log_log2 plain packets, each
    weighted by the L2 norm of its in-image contributions -- the density that minimises
    the summed pixel variance is proportional to that norm; logging and training time
    are added to every ladder point) and Philox MC, all on the wavefront tracer with FP64
    accumulation.  Every arm is randomized (Owen-scrambled Sobol with independent seeds,
    the learned warp applied to those points; Philox keys) and its error at N packets is
    estimated from `replicates` independent renders of N packets (_replicate_error): no
    converged reference is needed, so the ladder can reach the 1e-3 target.  A render
    of N > 2^31 packets is N / 2^31 independently scrambled point sets of 2^31 points
    (the upper half of each 2^32-point Sobol set), averaged."""
    import torch

    from paper_2406_15632_gb300 import qmcrt as Q
    from paper_2406_15632_gb300 import scenes as S

    prob = S.clumpy_problem(n=128)
    sc = Q.Scene(prob)
    chunk = 1 << chunk_log2
    scenes = {}

    def scene(gen, seed):
        if (gen, seed) not in scenes:
            scenes[(gen, seed)] = Q.Scene(prob.replace(generator=gen, seed=seed), grid_device=sc.grid)
        return scenes[(gen, seed)]

    # training: log 2^n_log_log2 plain packets (unscrambled Sobol, points 1 ..), minibatch
    # Adam on the log (2^20 to 2^23 logged packets, one to four epochs, learning rates
    # 3e-3 to 3e-2 all gave the same error at equal packets, within 3 %)
    n_log = 1 << n_log_log2
    log = torch.zeros((n_log, 5), dtype=torch.float32, device="cuda")
    logger = Q.LearnedTracer(sc, None, chunk=min(chunk, n_log), wavefront=True)
    _, ms_log = _timed(lambda: logger.trace(1, n_log, sc.accum_buffer("f64"), train_log=log))
    del logger
    W = Q.Warp(seed=2, uniform_mix=mix)
    xs, ws = log[:, :3].contiguous(), log[:, 4 if weight == "l2" else 3].contiguous()
    losses, ms_train = _timed(lambda: W.train(xs, ws, epochs=epochs, batch=1 << batch_log2, lr=lr))
    del log, xs, ws

    out = torch.empty((1, 3, prob.ny, prob.nx), dtype=torch.float64, device="cuda")
    tracers = {}

    def render(arm, rep, n):
        """One randomized render of n packets (replicate rep) and its wall time in ms."""
        gen = "philox" if arm == "mc_philox" else "sobol_owen"
        blocks = max(1, n >> SOBOL_BLOCK_LOG2) if gen == "sobol_owen" else 1
        per = n // blocks
        parts = [scene(gen, 1000 * (rep + 1) + 7 * b + (11 if arm == "mc_philox" else 0)) for b in range(blocks)]
        if arm not in tracers:  # one tracer (workspace) per arm, pointed at each scene in turn
            tracers[arm] = Q.LearnedTracer(sc, W if arm == "learned_qmc" else None, chunk=chunk, wavefront=True)
        tr = tracers[arm]
        buf = sc.accum_buffer("f64")

        def go():
            buf.zero_()
            for s in parts:
                tr.scene = s  # same grid, this point set's generator and seed
                tr.trace(per, per, buf)  # points per .. 2 per - 1: one whole net block
            sc.reduce(buf, 1.0 / n, accum="f64", out=out)
        _, ms = _timed(go)
        return out[0, 0].clone(), ms

    arms_ladder = {"plain_qmc": ladder, "learned_qmc": ladder, "mc_philox": mc_ladder or ladder}
    for arm in arms_ladder:
        render(arm, 0, 1 << 16)  # warm
    arms = {}
    for arm, lad in arms_ladder.items():
        rows = []
        for lg in lad:
            imgs, mss = [], []
            for r in range(replicates):
                img, ms = render(arm, r, 1 << lg)
                imgs.append(img)
                mss.append(ms)
            rows.append({"log2_n": lg, "ms": statistics.median(mss), "rms": _replicate_error(imgs)})
        arms[arm] = rows
        tracers.clear()
    overhead = {"learned_qmc": ms_log + ms_train}
    summary = _tte_summary(arms, targets, overhead, key="rms")
    for tgt, row in summary.items():
        p, l, m = (row[k]["ms"] for k in ("plain_qmc", "learned_qmc", "mc_philox"))
        row["learned_speedup_vs_plain"] = p / l if p and l else None
        row["plain_qmc_speedup_vs_mc"] = m / p if p and m else None
    return {"workload": "clumpy envelope 128^3 (radial tau 5, sigma 1 clumps), point source, 20 orders, forced, "
                        "roulette 1e-4, g 0.6, albedo 0.7, 512x512 I/Q/U, FP32 trace, FP64 accumulate",
            "error": f"RMS relative of the I image, estimated from {replicates} independent randomized renders "
                     "(Owen-scrambled Sobol seeds, Philox keys) at each N",
            "training": {"logged_packets": n_log, "log_ms": ms_log, "train_ms": ms_train, "epochs": epochs,
                         "batch": 1 << batch_log2, "lr": lr, "uniform_mix": mix, "sample_weight": weight,
                         "loss_first": losses[0], "loss_last": sum(losses[-8:]) / len(losses[-8:]),
                         "warp_error_flag": int(W.error.item())},
            "ladder": arms, "time_to_error_ms": summary}


def run_time_to_error_disk(ladder=(20, 22, 24, 26), ref_log2=28, ref_seeds=(101, 102, 103, 104)):
    return run_time_to_error_qmc(workload_problem(), "flared disk 256^3 single scattering, point source, "
                                 "theta 45 deg, 256x256 I/Q/U, FP32 trace, int64 accumulate", ladder, ref_log2, ref_seeds)


def run_time_to_error_geometries(ladder=(20, 22, 24, 26), ref_log2=27, ref_seeds=(101, 102, 103, 104)):
    """The paper's other test geometries (Sec. 5) through the same comparison: the disk
    seen from the pole, the dust shell and the fractal cloud."""
    from paper_2406_15632_gb300 import scenes as S

    cases = {"disk_pole": (workload_problem().replace(theta_obs=0.0), "flared disk 256^3 seen from the pole"),
             "shell": (S.shell_envelope_problem(), "dust shell 256^3 (radial tau 0.1), pole-on"),
             "fractal": (S.fractal_cloud_problem(), "fractal cloud 200^3 (N 32, D 2.3, tau 2), theta 60 deg")}
    return {k: run_time_to_error_qmc(p, w, ladder, ref_log2, ref_seeds) for k, (p, w) in cases.items()}


def run_time_to_error_qmc(prob, workload, ladder=(20, 22, 24, 26), ref_log2=28, ref_seeds=(101, 102, 103, 104)):
    """The paper's comparison (Sec. 6) on one single-scattering problem: wall time to a
    fixed image error for Sobol, Owen-scrambled Sobol, Niederreiter, Faure, Halton,
    Hammersley (its own set of N points for every N) and Philox MC, all through the same
    FP32 tracer with fixed-point accumulation, against an Owen-scrambled reference."""
    import torch

    from paper_2406_15632_gb300 import qmcrt as Q

    base = Q.Scene(prob)
    ref, ref_err, ref_n = _reference_image(Q, prob, base.grid, ref_log2, ref_seeds, "i64")

    def renderer(gen, seed=0):
        out = torch.empty((1, 3, prob.ny, prob.nx), dtype=torch.float64, device="cuda")

        def render(n):
            p = prob.replace(generator=gen, seed=seed, total_n=n if gen == "hammersley" else 0)
            s = Q.Scene(p, grid_device=base.grid)
            fb = Q.default_frac_bits(p, n)
            buf = s.accum_buffer("i64")
            first = 1 if gen == "hammersley" else n

            def go():
                s.trace(first, n, buf, frac_bits=fb)
                s.reduce(buf, 1.0 / n, frac_bits=fb, out=out)
            _, ms = _timed(go)
            return out[0, 0].clone(), ms
        return render

    gens = {"sobol": ("sobol", 0), "sobol_owen": ("sobol_owen", 1), "niederreiter": ("niederreiter", 0),
            "faure": ("faure", 0), "halton": ("halton", 0), "hammersley": ("hammersley", 0),
            "mc_philox": ("philox", 7)}
    for g, sd in gens.values():
        renderer(g, sd)(1 << 16)
    arms = {k: _ladder(renderer(g, sd), ladder, ref, ref_err) for k, (g, sd) in gens.items()}
    summary = _tte_summary(arms, (0.05, 0.02, 1e-2, 3e-3))
    for tgt, row in summary.items():
        m = row["mc_philox"]["ms"]
        for k in gens:
            if k != "mc_philox" and row[k]["ms"] and m:
                row[k]["speedup_vs_mc"] = m / row[k]["ms"]
    return {"workload": workload,
            "error": "RMS relative of the I image (L1 relative, the paper's norm, also listed)",
            "reference": {"packets": ref_n, "generator": "sobol_owen", "seeds": list(ref_seeds),
                          "estimated_rms_error": ref_err},
            "ladder": arms, "time_to_error_ms": summary}


def _sig(x, digits=4):
    """x rounded to `digits` significant digits (None stays None)."""
    if x is None or isinstance(x, bool) or not isinstance(x, (int, float)) or x == 0 or not math.isfinite(x):
        return x
    return round(x, digits - 1 - int(math.floor(math.log10(abs(x)))))


def _speedups(tte, num, den, targets=None):
    """{target: time(num) / time(den)} over the targets where both arms have a time, and
    the targets where either time was extrapolated beyond its ladder."""
    out, extrap = {}, []
    for tgt, row in tte.items():
        if targets and tgt not in targets:
            continue
        a, b = row.get(num, {}), row.get(den, {})
        if a.get("ms") and b.get("ms"):
            out[tgt] = _sig(a["ms"] / b["ms"], 3)
            if a.get("extrapolated") or b.get("extrapolated"):
                extrap.append(tgt)
    return out, extrap


def summarize(sections):
    """One or two numbers per detailed section, for the headline line; `extrapolated`
    lists the time-to-error speedups taken beyond a ladder's last point."""
    out, extrap = {}, []
    ms = sections.get("multiple_scattering")
    if ms:
        out["multiple_scattering"] = {"packets_per_s": _sig(ms["packets_per_s"]), "frac": _sig(ms["roofline"]["frac"], 3)}
    b = sections.get("batched")
    if b:
        out["batched"] = {"packets_per_s": _sig(b["packets_per_s"]), "vs_each": _sig(b["speedup_at_equal_images"], 3)}
        if "time_to_error" in b:
            out["batched"]["tte_speedup"] = _sig(b["time_to_error"].get("speedup"), 3)
    o = sections.get("observers")
    if o:
        out["observers_speedup"] = _sig(o["speedup"], 3)
    le = sections.get("time_to_error_learned_vs_plain")
    if le:
        sp, ex = _speedups(le["time_to_error_ms"], "plain_qmc", "learned_qmc")
        out["learned_vs_plain_at_rms"] = sp
        extrap += [f"learned@{t}" for t in ex]
    d = sections.get("time_to_error_qmc_vs_mc_disk")
    if d:
        sp, ex = _speedups(d["time_to_error_ms"], "mc_philox", "sobol", ("0.01", "0.003"))
        out["sobol_vs_mc_at_rms"] = sp
        extrap += [f"sobol@{t}" for t in ex]
    if extrap:
        out["extrapolated"] = extrap
    return out


def headline(line, sections):
    """The compact last line: the contract's keys, the roofline, e2e, clocks, the CPU
    baseline and a summary of the detailed sections (printed on earlier lines)."""
    h = {k: line[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
                              "gpu_launches") if k in line}
    h["value"] = _sig(h["value"], 6)
    h["ms_per_step"] = _sig(h["ms_per_step"], 6)
    h["roofline"] = {k: _sig(line["roofline"].get(k), 4) for k in ("bound", "achieved", "peak", "unit", "frac",
                                                                    "traffic", "kernel")}
    h["e2e"] = {k: _sig(v, 6) for k, v in h["e2e"].items()}
    clk = line.get("clocks") or {}
    h["clocks"] = {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    cb = sections.get("cpu_baseline")
    if cb:
        h["cpu_baseline"] = {"value": _sig(cb["value"]), "unit": cb["unit"], "cores": cb["cores"], "kind": cb["kind"],
                             "sample": cb["sample_short"], "one_core": _sig(cb["single_core"]["value"])}
    s = summarize(sections)
    if s:
        h["sections"] = s
    return h


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
    ap.add_argument("--tte-c5", action="store_true",
                    help="only the learned-vs-plain time to error at the clumpy workload's 1e-3 target (a long run: "
                         "ladders to 2^35 packets, training on 2^22 logged packets); prints that section")
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
    if args.tte_c5:
        res = run_time_to_error_learned(ladder=(20, 22, 24, 26, 28, 30, 32, 34, 35), mc_ladder=(20, 22, 24, 26, 28, 30),
                                        n_log_log2=22, chunk_log2=24)
        print(json.dumps({"section": "time_to_error_learned_vs_plain_c5", **res}), flush=True)
        return 0
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
    # the tracer skips, from one lookup of the bound map, the rays that cannot scatter,
    # resumes each march from a boundary of the first walk and ends each peel-off walk on
    # the tail map: its algorithmic work is the oracle's count of the other rays' walks with
    # each cell of a ray walked once and the peel-offs' cells whose depth can matter
    cpp = cells_per_packet(key="cells_per_packet_scattering_rays_single_pass_tail")
    kern_avg_s = kern_total / args.steps / 1e3
    achieved_ops = n * (cpp * OPS_PER_CELL + OPS_PER_PACKET) / kern_avg_s
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "packets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(n),
        "roofline": {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": achieved_ops / peak_ops, "traffic": traffic,
                     "kernel": "k_trace_single<float>", "kernel_ms": kern_avg_s * 1e3,
                     "per_unit": f"{OPS_PER_CELL} ops per cell visit x {cpp:.2f} cells per packet (oracle count "
                                 f"of the walks of rays with tau_1 >= tau_min, without the march's second pass and "
                                 f"the peel-off cells past a remaining depth of 2^-24) "
                                 f"+ {OPS_PER_PACKET} ops of setup per packet",
                     "peak_basis": f"{SMS} SMs x {LANES_PER_SM} lanes x {max_mhz:.0f} MHz (measured max clock)"},
        "e2e": {"value": e2e_value, "unit": "packets/s", "h2d_bytes_per_step": R.input_bytes(),
                "d2h_bytes_per_step": R.output_bytes()},
        "gpu_launches": 2 * args.steps * 1,
        "clocks": clk,
    }
    # Detailed sections go on their own lines first; the last line of stdout is the
    # compact headline (a few hundred bytes), which is what a reader of the tail parses.
    sections = {}

    def section(name, fn):
        sections[name] = fn()
        print(json.dumps({"section": name, **sections[name]}), flush=True)
    if world == 1 and not args.no_extras:
        section("multiple_scattering", run_multiple_scattering)
        section("batched", run_batched)
        section("observers", run_observers)
        section("time_to_error_learned_vs_plain", run_time_to_error_learned)
        section("time_to_error_qmc_vs_mc_disk", run_time_to_error_disk)
        for k, v in run_time_to_error_geometries().items():
            sections[f"time_to_error_qmc_vs_mc_{k}"] = v
            print(json.dumps({"section": f"time_to_error_qmc_vs_mc_{k}", **v}), flush=True)
    if world == 1 and not args.no_cpu_baseline:
        section("cpu_baseline", run_cpu_baseline)
    print(json.dumps(headline(line, sections), separators=(",", ":")), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
