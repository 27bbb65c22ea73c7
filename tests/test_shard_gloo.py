"""Multi-rank path on CPU (gloo, world size 2): packet ranges partition the point set,
step blocks never overlap, and the summed per-rank images equal one unsharded run."""
import os
import socket

import numpy as np
import pytest

from paper_2406_15632_gb300 import shard


def test_split_range_partitions_exactly():
    for count in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [shard.split_range(5, count, r, world) for r in range(world)]
            nxt = 5
            for f, c in parts:
                assert f == nxt and c >= 0
                nxt = f + c
            assert nxt == 5 + count


def test_step_blocks_are_disjoint_and_below_2_32():
    n = 1 << 24
    nb = (1 << 32) // n - 1
    seen = set()
    for step in range(30):
        for r in range(8):
            f = shard.step_range(step, r, 8, n, nb)
            assert f >= 1 and f + n - 1 < 1 << 32
            if step * 8 + r < nb:
                assert f not in seen
                seen.add(f)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, N, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_2406_15632_gb300 import scenes as S

    prob = S.flared_disk_problem(n=32, nx=32, ny=32)
    first, count = shard.split_range(1, N, rank, world)
    img = torch.from_numpy(O.trace_single(prob, first, count, nthreads=1))
    shard.allreduce_image(img)
    ints = torch.full((4,), rank + 1, dtype=torch.int64) * (1 << 40)
    shard.allreduce_image(ints)
    if rank == 0:
        q.put((img.numpy(), ints.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_sum_to_the_unsharded_image():
    import torch.multiprocessing as mp

    from oracle import oracle as O
    from paper_2406_15632_gb300 import scenes as S

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    N = 5000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, N, q)) for r in range(2)]
    for p in procs:
        p.start()
    img, ints = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = O.trace_single(S.flared_disk_problem(n=32, nx=32, ny=32), 1, N, nthreads=1)
    assert np.allclose(img, ref, rtol=1e-12, atol=1e-300)
    assert np.all(ints == 3 * (1 << 40))
