"""The argument behind the tail map of an observer direction (qmcrt_tail_map), checked on the
CPU: a numpy model of its slab recurrence (4^3-cell blocks, slabs across the axis the
direction crosses fastest, lateral reach counted in cells) bounds the optical depth the
oracle integrates from any point of a cell along the direction to the edge of the grid, for
grids of unequal cells holding a few dense boxes (where the bound is tight, so a lateral
reach, a slab path or a slab axis taken too small shows) and random, axis-parallel and tied
directions."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

BLOCK = 4


def slab_bound(grid, lo, hi, k):
    """Per cell [nz][ny][nx]: the model's bound on the depth ahead along unit k."""
    nz, ny, nx = grid.shape
    n = np.array([nx, ny, nz])
    h = (np.array(hi) - np.array(lo)) / n
    nb = (n + BLOCK - 1) // BLOCK
    Kb = np.zeros((nb[2], nb[1], nb[0]))
    g = np.maximum(grid, 0.0)
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                Kb[bz, by, bx] = g[BLOCK * bz:BLOCK * (bz + 1), BLOCK * by:BLOCK * (by + 1),
                                   BLOCK * bx:BLOCK * (bx + 1)].max()
    speed = np.abs(k) / h
    a = int(np.argmax(speed))
    lat = [q for q in range(3) if q != a]
    sgn = np.sign(k).astype(int)

    def reach(q):
        if k[q] == 0.0:
            return 1
        r = speed[q] / speed[a] * (1.0 + 1e-9)
        return 1 + ((BLOCK - 1) + math.floor(BLOCK * r) + 2) // BLOCK

    L = {q: reach(q) for q in lat}
    path = BLOCK * h[a] / abs(k[a]) * (1.0 + 1e-6)
    Kt = Kb.transpose(2, 1, 0)  # [x][y][z] indexing by axis number
    B = np.zeros_like(Kt)
    order = range(nb[a] - 1, -1, -1) if sgn[a] > 0 else range(nb[a])
    prev = None
    for j in order:
        cur = np.zeros([nb[q] for q in lat])
        for ib in range(nb[lat[0]]):
            for ic in range(nb[lat[1]]):
                kmax = nmax = 0.0
                for ob in range(L[lat[0]]):
                    qb = ib + sgn[lat[0]] * ob
                    if not 0 <= qb < nb[lat[0]]:
                        continue
                    for oc in range(L[lat[1]]):
                        qc = ic + sgn[lat[1]] * oc
                        if not 0 <= qc < nb[lat[1]]:
                            continue
                        idx = [0, 0, 0]
                        idx[a], idx[lat[0]], idx[lat[1]] = j, qb, qc
                        kmax = max(kmax, Kt[tuple(idx)])
                        if prev is not None:
                            nmax = max(nmax, prev[qb, qc])
                cur[ib, ic] = kmax * path + nmax
                idx = [0, 0, 0]
                idx[a], idx[lat[0]], idx[lat[1]] = j, ib, ic
                B[tuple(idx)] = cur[ib, ic]
        prev = cur
    cells = B.transpose(2, 1, 0)  # back to [z][y][x] of blocks
    return np.repeat(np.repeat(np.repeat(cells, BLOCK, 0), BLOCK, 1), BLOCK, 2)[:nz, :ny, :nx]


def _directions(rng):
    out = [(1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0), (math.sqrt(0.5), 0.0, math.sqrt(0.5)),
           (-1.0, 1.0, 1.0), (1.0, 1.0, -1e-7)]
    for _ in range(6):
        out.append(tuple(rng.normal(size=3)))
    return [np.array(d) / np.linalg.norm(d) for d in out]


def _blobs(rng, shape):
    """A few dense boxes of cells in an empty grid: the bound is tight only where the blocks
    a ray can reach are counted right."""
    g = np.zeros(shape, dtype=np.float32)
    for _ in range(3):
        size = rng.integers(1, 7, size=3)
        at = rng.integers(0, np.maximum(np.array(shape) - size, 0) + 1)
        g[at[0]:at[0] + size[0], at[1]:at[1] + size[1], at[2]:at[2] + size[2]] = rng.uniform(0.5, 4.0)
    return g


@pytest.mark.parametrize("seed", range(8))
def test_slab_bound_holds_for_the_oracle(seed):
    rng = np.random.default_rng(seed)
    shape = (int(rng.integers(8, 17)), int(rng.integers(8, 17)), int(rng.integers(8, 17)))
    grid = _blobs(rng, shape)
    lo = tuple(rng.uniform(-1.5, -0.5, size=3))
    hi = tuple(np.array(lo) + rng.uniform(0.8, 2.5, size=3))
    prob = S.Problem(grid=grid, lo=lo, hi=hi)
    nz, ny, nx = shape
    h = (np.array(hi) - np.array(lo)) / np.array([nx, ny, nz])
    for k in _directions(rng):
        bound = slab_bound(grid.astype(np.float64), lo, hi, k)
        for _ in range(200):
            c = rng.integers(0, [nx, ny, nz])
            off = np.where(rng.uniform(size=3) < 0.5, rng.choice([1e-6, 1 - 1e-6], size=3), rng.uniform(size=3))
            p = np.array(lo) + (c + off) * h
            tau = O.tau_ray(prob, p, k)
            assert tau <= bound[c[2], c[1], c[0]] * (1 + 1e-9) + 1e-300, (seed, k, c, tau)
