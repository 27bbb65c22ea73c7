"""Pins of the oracle's optical-depth integration and march (Sec. 3.4): closed-form
chords through homogeneous media, exact cell sums along axis-aligned rays, and a
fine midpoint-rule integration along random rays through random grids."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S


def box_exit_distance(p, d, lo=-1.0, hi=1.0):
    t = np.inf
    for a in range(3):
        if d[a] > 0:
            t = min(t, (hi - p[a]) / d[a])
        elif d[a] < 0:
            t = min(t, (lo - p[a]) / d[a])
    return t


def midpoint_tau(grid, p, d, t_end, steps=400_000, lo=-1.0, hi=1.0):
    """Independent reference: sample the cell value at midpoints of a fine subdivision."""
    n = grid.shape[0]
    t = (np.arange(steps) + 0.5) * (t_end / steps)
    x = p[None, :] + t[:, None] * d[None, :]
    idx = np.clip(np.floor((x - lo) / (hi - lo) * n).astype(int), 0, n - 1)
    vals = grid[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
    return vals.sum() * (t_end / steps)


def random_unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def test_homogeneous_grid_tau_is_k_times_chord():
    rng = np.random.default_rng(1)
    prob = S.Problem(grid=S.homogeneous_grid(8, 0.7))
    for _ in range(200):
        p = rng.uniform(-0.99, 0.99, 3)
        d = random_unit(rng)
        tau = O.tau_ray(prob, p, d)
        k = float(np.float32(0.7))  # the grid stores single-precision cells
        assert tau == pytest.approx(k * box_exit_distance(p, d), rel=1e-13, abs=1e-15)


def test_axis_aligned_rays_sum_cells_exactly():
    g = S.random_grid(6, seed=3)
    prob = S.Problem(grid=g)
    h = 2.0 / 6
    for j in range(6):
        for l in range(6):
            p = np.array([-1.0, -1.0 + (j + 0.5) * h, -1.0 + (l + 0.5) * h])
            tau = O.tau_ray(prob, p, [1.0, 0.0, 0.0])
            ref = g[l, j, :].astype(np.float64).sum() * h
            assert tau == pytest.approx(ref, rel=1e-14)
            # the same row backwards from the far face
            p2 = p.copy()
            p2[0] = 1.0
            assert O.tau_ray(prob, p2, [-1.0, 0.0, 0.0]) == pytest.approx(ref, rel=1e-14)


def test_random_rays_match_midpoint_integration():
    rng = np.random.default_rng(7)
    g = S.random_grid(5, seed=11)
    prob = S.Problem(grid=g)
    for _ in range(25):
        p = rng.uniform(-0.9, 0.9, 3)
        d = random_unit(rng)
        t_end = box_exit_distance(p, d)
        ref = midpoint_tau(g, p, d, t_end)
        assert O.tau_ray(prob, p, d) == pytest.approx(ref, rel=2e-4)


def test_ray_from_cell_corner_and_face():
    """Start exactly on faces and edges: the start cell is the one the ray enters."""
    g = S.random_grid(4, seed=5)
    prob = S.Problem(grid=g)
    rng = np.random.default_rng(2)
    for _ in range(50):
        p = np.round(rng.uniform(-1, 1, 3) * 2) / 2  # on the cell lattice of n=4
        d = random_unit(rng)
        t_end = box_exit_distance(p, d)
        if t_end <= 0:
            continue
        ref = midpoint_tau(g, p + 1e-12 * d, d, t_end)
        assert O.tau_ray(prob, p, d) == pytest.approx(ref, rel=2e-4, abs=1e-9)


def test_march_reaches_requested_depth():
    rng = np.random.default_rng(9)
    g = S.random_grid(5, seed=13)
    prob = S.Problem(grid=g)
    for _ in range(25):
        p = rng.uniform(-0.8, 0.8, 3)
        d = random_unit(rng)
        total = O.tau_ray(prob, p, d)
        tau = rng.uniform(0.05, 0.95) * total
        hit, q = O.march_ray(prob, p, d, tau)
        assert hit
        t = np.dot(q - p, d)
        assert np.allclose(q, p + t * d, atol=1e-14)
        assert midpoint_tau(g, p, d, t) == pytest.approx(tau, rel=2e-4)
        # beyond the total optical depth the packet leaves the grid
        hit2, _ = O.march_ray(prob, p, d, total * 1.01 + 1e-9)
        assert not hit2


def test_march_in_homogeneous_sphere_is_tau_over_k():
    prob = S.homogeneous_sphere_problem()
    rng = np.random.default_rng(4)
    for _ in range(50):
        d = random_unit(rng)
        p = rng.uniform(-0.5, 0.5, 3)
        hit, q = O.march_ray(prob, p, d, 0.03)
        assert hit
        assert np.allclose(q, p + (0.03 / 0.1) * d, atol=1e-14)


def test_sphere_chord_closed_form():
    prob = S.homogeneous_sphere_problem()
    for r in (0.0, 0.3, 0.9):
        for mu in (-1.0, -0.4, 0.0, 0.7, 1.0):
            p = np.array([0.0, 0.0, r])
            d = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
            s = -r * mu + math.sqrt(1 - r * r * (1 - mu * mu))
            assert O.tau_ray(prob, p, d) == pytest.approx(0.1 * s, rel=1e-14, abs=1e-16)


def test_flared_disk_grid_radial_tau_follows_density_law():
    """Along x at the height z of the first cell centre above the midplane, the grid's
    optical depth follows the integral of the disk law (1 at z = 0) to the accuracy of
    the cell-centre sampling."""
    quad = pytest.importorskip("scipy.integrate").quad
    assert quad(lambda r: r ** -2 / 9.0, 0.1, 1.0)[0] == pytest.approx(1.0, rel=1e-12)
    for n in (128, 256):
        g = S.flared_disk_grid(n)
        prob = S.Problem(grid=g)
        hc = 2.0 / n
        z = 0.5 * hc
        tau = O.tau_ray(prob, [0.0, z, z], [1.0, 0.0, 0.0])
        ref = quad(lambda r: r ** -2 / 9.0 * math.exp(-0.5 * (z / (0.1 * r ** 1.25)) ** 2), 0.1, 1.0,
                   limit=200)[0]
        assert tau == pytest.approx(ref, rel=0.04)


def test_clumpy_grid_mean_radial_tau_is_five():
    g = S.clumpy_envelope_grid(64)
    prob = S.Problem(grid=g)
    rng = np.random.default_rng(0)
    taus = [O.tau_ray(prob, [0.0, 0.0, 0.0], random_unit(rng)) for _ in range(400)]
    assert np.mean(taus) == pytest.approx(5.0, rel=0.25)


def test_ray_cells_counts_the_cells_a_tolerance_leaves_out():
    """Along a row of known cells: the walk from the middle of cell 1 visits cells 1..7;
    with a tolerance it may leave out the trailing cells whose depths sum to at most it."""
    n = 8
    h = 2.0 / n
    g = np.zeros((n, n, n), dtype=np.float32)
    g[3, 3, :] = [5.0, 2.0, 0.0, 3.0, 1e-9, 0.0, 0.0, 0.0]
    prob = S.Problem(grid=g)
    p = [-1.0 + 1.5 * h, -1.0 + 3.5 * h, -1.0 + 3.5 * h]
    d = [1.0, 0.0, 0.0]
    depths = [2.0 * h / 2, 0.0, 3.0 * h, 1e-9 * h, 0.0, 0.0, 0.0]
    assert O.tau_ray(prob, p, d) == pytest.approx(sum(depths), rel=1e-6)
    for eps, needed in ((0.0, 4), (1.01e-9 * h, 3), (0.99e-9 * h, 4), (3.0 * h * 1.0001, 1), (10.0, 0)):
        assert O.ray_cells(prob, [p], d, eps).tolist() == [[7, needed]], eps
