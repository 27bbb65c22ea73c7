"""Run one named workload of the library once, on cuda:0, and print its wall time.

    python -m paper_2406_15632_gb300.workloads <name> [--log2-n L] [--repeat R]

Names:
  disk_single      single scattering, 256^3 flared disk (--grid G: G^3), 256x256 I/Q/U, FP32, 2^L packets
  star_single      the same disk lit by the finite limb-darkened star (inverse order), 2^L packets
  clumpy_multiple  multiple scattering (20 orders), 128^3 clumpy envelope, 512x512, 2^L packets
  clumpy_wavefront the same packets order by order (live packets regrouped between orders)
  warp_forward     fused forward of the learned warp on 2^L Sobol points
  warp_train       one epoch of minibatch training (2^16 rows per step) on 2^L samples
  batch            the 256-instance finite-star batch in one persistent launch (graph replay)

Each run is preceded by one warm-up run.  Used to time a single kernel family in
isolation and as the command under a profiler.
"""
from __future__ import annotations

import argparse
import sys
import time


def _cuda_ms(fn, repeat):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(repeat):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / repeat


def main(argv=None) -> int:
    import torch

    from . import qmcrt as Q
    from . import scenes as S

    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=["disk_single", "star_single", "clumpy_multiple", "clumpy_wavefront",
                                     "warp_forward", "warp_train", "batch"])
    ap.add_argument("--log2-n", type=int, default=20)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--instances", type=int, default=0, help="batch: the first N instances only (0: all 256)")
    ap.add_argument("--grid", type=int, default=0, help="disk_single: cells per axis of the disk (0: 256)")
    a = ap.parse_args(argv)
    Q.load()
    n = 1 << a.log2_n
    t0 = time.perf_counter()
    if a.name in ("disk_single", "star_single", "clumpy_multiple"):
        prob = {"disk_single": lambda: S.flared_disk_problem(n=a.grid or 256),
                "star_single": lambda: S.finite_star_disk_problem(n=a.grid or 256),
                "clumpy_multiple": lambda: S.clumpy_problem(n=128)}[a.name]()
        sc = Q.Scene(prob)
        fb = Q.default_frac_bits(prob, n)
        buf = sc.accum_buffer("i64")

        def run():
            buf.zero_()
            sc.trace(n, n, buf, frac_bits=fb)
        ms = _cuda_ms(run, a.repeat)
    elif a.name == "clumpy_wavefront":
        prob = S.clumpy_problem(n=128)
        sc = Q.Scene(prob)
        fb = Q.default_frac_bits(prob, n)
        buf = sc.accum_buffer("i64")
        ws = sc.wavefront_workspace(n)

        def run():
            buf.zero_()
            sc.trace_wavefront(n, n, buf, ws, frac_bits=fb)
        ms = _cuda_ms(run, a.repeat)
    elif a.name == "warp_forward":
        W = Q.Warp(seed=1, uniform_mix=0.1)
        u = Q.generate_points("sobol", 3, 1, n, "f32")
        x = torch.empty((n, 3), device="cuda")
        lj = torch.empty(n, device="cuda")
        ms = _cuda_ms(lambda: W.forward_into(u, x, lj), a.repeat)
    elif a.name == "warp_train":
        W = Q.Warp(seed=1, uniform_mix=0.1)
        xs = Q.generate_points("sobol", 3, 1, n, "f32")
        ws = torch.ones(n, device="cuda")
        ms = _cuda_ms(lambda: W.train(xs, ws, epochs=1, batch=min(n, 1 << 16), lr=1e-3), a.repeat)
    else:
        prob = S.finite_star_disk_problem(n=256)
        inst = S.batched_instances()
        if a.instances > 0:
            inst = inst[: a.instances]
        B = Q.Batch(prob, inst, chunk_log2=24, block_size=256, ctas_per_sm=0, packets_per_thread=1)
        B.capture()
        ms = _cuda_ms(B.replay, a.repeat)
    print(f"{a.name} log2_n={a.log2_n}: {ms:.3f} ms per run ({time.perf_counter() - t0:.1f} s wall)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
