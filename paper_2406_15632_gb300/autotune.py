"""Autotuner for the batched persistent launch.

Chooses the work decomposition of qmcrt_trace_batch (largest chunk, CTA size, resident
CTAs per SM, packets per thread per work tile) by timing graph replays of a
stratified subset of the batch (every stride-th instance by budget, full budgets) with
CUDA events, and caches the winner per device and workload signature in
_build/autotune.json.  The decomposition never changes the images (fixed-point sums
are order-independent), only the time.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import qmcrt as Q

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

DEFAULT_SPACE = {
    "chunk_log2": (18, 20, 24),
    "block_size": (128, 256),
    "ctas_per_sm": (0, 3),
    "packets_per_thread": (1, 2, 4),
}


def signature(prob, instances, precision) -> str:
    h = hashlib.sha256()
    h.update(repr((prob.source, prob.emit_order, prob.generator, prob.nx, prob.ny, prob.splat, precision,
                   None if prob.grid is None else prob.grid.shape)).encode())
    h.update(repr([(round(I.theta_obs, 6), round(I.g, 6), round(I.kscale, 6), I.n_packets) for I in instances]).encode())
    return h.hexdigest()[:16]


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)


def time_batch(batch, repeats: int = 3) -> float:
    """Milliseconds per graph replay (median of repeats, after one warm replay)."""
    import torch

    batch.capture()
    batch.replay()
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.replay()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return sorted(times)[len(times) // 2]


def tune_batch(prob, instances, *, precision: str = "f32", stride: int = 8, space: dict | None = None,
               use_cache: bool = True, scene=None) -> dict:
    """Best batch configuration {chunk_log2, block_size, ctas_per_sm, packets_per_thread}
    for this workload on this device.  Timed on every stride-th instance with its full
    budget (chunk coherence depends on the budget, so budgets are not scaled down)."""
    import torch

    space = space or DEFAULT_SPACE
    key = f"{torch.cuda.get_device_name()}|{signature(prob, instances, precision)}|{stride}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    subset = sorted(instances, key=lambda I: I.n_packets)[::stride]
    batch = Q.Batch(prob, subset, precision=precision, scene=scene)
    table = []
    for cfg in itertools.product(*space.values()):
        c = dict(zip(space.keys(), cfg))
        batch.set_config(**c)
        table.append((time_batch(batch), c))
    table.sort(key=lambda x: x[0])
    best = dict(table[0][1], ms=table[0][0], tried=len(table), worst_ms=table[-1][0])
    cache[key] = best
    if use_cache:
        _store_cache(cache)
    return best
