"""Scene generators: the fractal cloud (the paper's third geometry, Sec. 5) and the
normalisation of its density to an average radial optical depth, checked with the
oracle's own optical-depth walk."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S


def test_fractal_points_count_range_and_clumping():
    N, levels = 16, 3
    pts = S.fractal_cloud_points(N=N, D=2.3, levels=levels, seed=7)
    assert pts.shape == (N ** levels, 3)
    assert np.all((pts >= 0) & (pts < 1))
    # last-generation points sit in cubes of edge (2 N^(1/D))^-(levels-1) around their
    # parents: their nearest neighbours are far closer than for uniform points
    rng = np.random.default_rng(0)
    sample = pts[rng.choice(len(pts), 300, replace=False)]
    d = np.sqrt(((sample[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    d[d == 0] = np.inf
    nn = d.min(axis=1)
    uniform_nn = 0.55 * len(pts) ** (-1 / 3)  # mean nearest-neighbour distance of uniform points
    assert np.median(nn) < 0.3 * uniform_nn


def test_fractal_grid_average_radial_tau_matches_oracle_walk():
    """The generator normalises the mean, over a seeded set of directions, of the
    optical depth from the centre to the surface; the oracle's cell walk over the same
    directions gives the same mean."""
    n, tau, seed, dirs = 40, 2.0, 11, 256
    grid = S.fractal_cloud_grid(n=n, N=12, D=2.3, levels=3, tau=tau, seed=seed, directions=dirs)
    rng = np.random.Generator(np.random.Philox(seed + 1))
    v = rng.normal(size=(dirs, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    prob = S.Problem(grid=grid)
    taus = [O.tau_ray(prob, [0.0, 0.0, 0.0], d) for d in v]
    assert np.mean(taus) == pytest.approx(tau, rel=1e-5)
    assert (grid > 0).mean() < 0.5  # clumped: most cells empty


def test_fractal_problem_defaults():
    p = S.fractal_cloud_problem(n=40)
    assert p.grid.shape == (40, 40, 40) and p.theta_obs == pytest.approx(math.radians(60))


def test_shell_envelope_radial_tau():
    """Along any ray from the centre the shell adds k (r_out - r_in) = tau, up to the
    cell sampling of the shell's two spheres."""
    grid = S.shell_envelope_grid(n=128, tau=0.1)
    prob = S.Problem(grid=grid)
    rng = np.random.default_rng(3)
    v = rng.normal(size=(64, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    taus = np.array([O.tau_ray(prob, [0.0, 0.0, 0.0], d) for d in v])
    assert np.mean(taus) == pytest.approx(0.1, rel=0.08)
