"""Packet-range sharding across ranks and the one exchange step (the image sum).

Packets are independent and point i is a pure function of i, so rank r of a world
of size W traces its own index range; the fixed-point images are then summed with
one all-reduce.  Integer sums are exact and order-independent, so any sharding gives
bit-for-bit the image of one unsharded run.
"""
from __future__ import annotations


def step_range(step: int, rank: int, world: int, n: int, n_blocks: int) -> int:
    """First point index of the n-packet block traced by `rank` at `step`: blocks of n
    consecutive indices starting at multiples of n from n on (index 0 is never used), so
    a power-of-two n is one whole net block of the sequence; assigned round-robin over
    (step, rank), wrapping after n_blocks blocks so every index stays below 2^32 (n_blocks
    at most 2^32 / n - 1)."""
    b = (step * world + rank) % n_blocks
    return (1 + b) * n


def split_range(first: int, count: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share of [first, first+count) for rank (sizes differ by at most 1)."""
    a = count * rank // world
    b = count * (rank + 1) // world
    return first + a, b - a


def allreduce_image(buf, group=None) -> None:
    """Sum the accumulation buffers of all ranks in place (the image exchange step)."""
    import torch.distributed as dist

    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
