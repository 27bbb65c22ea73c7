"""The bound map of rays from the source (qmcrt_sky_bound): it bounds the optical depth
the oracle integrates along every ray from the source (the origin, or the surface of a
star), and a trace that uses it to skip rays that cannot scatter gives the same image as
one that walks them."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def texel(d, m):
    """Face and texel of direction d in the cube map of the header's convention."""
    a = int(np.argmax(np.abs(d)))  # ties to the lower axis
    w = abs(d[a])
    u, v = [d[b] for b in range(3) if b != a]
    f = 2 * a + (1 if d[a] < 0 else 0)
    iu = min(m - 1, max(0, math.floor((u / w + 1) * 0.5 * m)))
    iv = min(m - 1, max(0, math.floor((v / w + 1) * 0.5 * m)))
    return f, iv, iu


def _directions(rng, n):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    special = [[1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 1, 0], [1, -1, 1], [0.6, 0.8, 0], [-1, 1, 1], [1e-7, 1, -1]]
    s = np.array(special, dtype=np.float64)
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    return np.concatenate([s, d])


@pytest.mark.parametrize("name", ["disk", "fractal", "random", "star"])
def test_map_bounds_the_oracle_optical_depth(Q, name):
    """Rays from the source (the origin, or points on the star's surface) never carry more
    optical depth, by the oracle's walk, than their direction's texel holds."""
    import torch

    prob = {"disk": S.flared_disk_problem(n=64), "fractal": S.fractal_cloud_problem(),
            "random": S.Problem(grid=S.random_grid(9, seed=5) * (S.random_grid(9, seed=6) > 1.2)),
            "star": S.finite_star_disk_problem(n=64, star_r=0.2)}[name]  # a star of 6.4 cells
    sc = Q.Scene(prob, sky=128)
    torch.cuda.synchronize()
    sky = sc.sky.cpu().numpy()
    rng = np.random.default_rng(3)
    tight = 0
    for d in _directions(rng, 3000):
        p = np.zeros(3)
        if prob.source == "sphere":  # a start point anywhere on the star
            p = rng.normal(size=3)
            p *= prob.star_r / np.linalg.norm(p)
        tau = O.tau_ray(prob.replace(kscale=1.0), p, d)
        b = sky[texel(d, 128)]
        assert tau <= b * (1 + 1e-12) + 1e-300, (d, tau, b)
        tight += tau > 0.1 * b
    assert tight > 0 or name != "disk"


CASES = {
    "disk": S.flared_disk_problem(n=64, nx=48, ny=48),
    "star_inverse": S.finite_star_disk_problem(n=64, nx=48, ny=48),
    "star_direct": S.finite_star_disk_problem(n=64, nx=48, ny=48, emit_order="direct"),
    "disk_kscale_taumin": S.flared_disk_problem(n=64, nx=48, ny=48, kscale=0.37, tau_min=1e-6),
    "fractal": S.fractal_cloud_problem(nx=64, ny=64),
    "clumpy_multiple": S.clumpy_problem(n=32, max_orders=8, nx=48, ny=48),
}


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("name", list(CASES))
def test_skipping_unscatterable_rays_changes_no_image(Q, name, precision):
    import torch

    prob = CASES[name]
    N = 1 << 15
    fb = Q.default_frac_bits(prob, N)
    imgs = []
    for sky in (0, 256):
        sc = Q.Scene(prob, sky=sky)
        buf = sc.accum_buffer("i64")
        sc.trace(1, N, buf, frac_bits=fb, precision=precision)
        imgs.append(buf)
    torch.cuda.synchronize()
    assert torch.equal(imgs[0], imgs[1])


def test_map_certifies_most_rays_that_cannot_scatter(Q):
    """On the disk, most packets whose tau_1 is below tau_min are caught by one lookup.  (Over
    a finite star the map must hold for every start point on the star, whose neighbourhoods
    take in the disk's dense inner rim: it is correct there but certifies few rays.)"""
    import torch

    prob = S.flared_disk_problem(n=128)
    sc = Q.Scene(prob, sky=512)
    torch.cuda.synchronize()
    sky = sc.sky.cpu().numpy()
    N = 1 << 13
    _, log = O.trace_single(prob, 1, N, log=True)
    idle = np.where(log[:, 8] == 1)[0]
    assert len(idle) > 0.3 * N
    caught = 0
    for j in idle:
        _, d, _, _, _ = O.emit_packet(prob, int(j) + 1)
        caught += 2 * sky[texel(d, 512)] * prob.kscale < prob.tau_min
    assert caught >= 0.8 * len(idle), caught / len(idle)


def test_batched_finite_star_is_unchanged_by_the_map(Q):
    """The batch (finite star, per-instance opacity scale) skips with the instance's kscale."""
    import torch

    prob = S.finite_star_disk_problem(n=32, nx=24, ny=24)
    inst = [S.Instance(theta_obs=0.3 + 0.4 * k, albedo=0.5 + 0.1 * k, g=0.2 * k, kscale=[0.5, 1.0, 4.0][k],
                       n_packets=4096 << k, first_index=4096 << k) for k in range(3)]
    outs = []
    for sky in (0, 128):
        B = Q.Batch(prob, inst, scene=Q.Scene(prob, sky=sky), chunk_log2=12, frac_bits=40)
        B.run()
        torch.cuda.synchronize()
        outs.append(B.accum.clone())
    assert torch.equal(outs[0], outs[1])


def test_edge_cases_of_the_map(Q):
    """An empty grid (every ray skipped, nothing scattered), a single dense cell beside the
    source (rays through it walked, the rest skipped), tau_min = 0 (nothing may be skipped)
    and a coarse map whose texel cones are too wide for the grid (infinite bounds: every ray
    walked): each image equals the one traced without the map."""
    import torch

    one = np.zeros((16, 16, 16), dtype=np.float32)
    one[8, 8, 9] = 40.0  # the cell just above-right of the origin (a grid vertex)
    cases = [S.flared_disk_problem(n=16).replace(grid=np.zeros((16, 16, 16), dtype=np.float32)),
             S.Problem(grid=one, nx=24, ny=24),
             S.flared_disk_problem(n=32, nx=24, ny=24, tau_min=0.0),
             S.flared_disk_problem(n=64, nx=24, ny=24)]
    for prob, sky in zip(cases, (64, 64, 64, 8)):
        N = 1 << 13
        fb = Q.default_frac_bits(prob, N)
        imgs = []
        for m in (0, sky):
            sc = Q.Scene(prob, sky=m)
            buf = sc.accum_buffer("i64")
            sc.trace(1, N, buf, frac_bits=fb)
            imgs.append(buf)
        torch.cuda.synchronize()
        assert torch.equal(imgs[0], imgs[1])
        if sky == 8:  # 8 texels per face edge over 64 cells: every texel's cone is too wide
            assert torch.isinf(Q.Scene(prob, sky=8).sky).all()
    sc = Q.Scene(cases[0], sky=64)
    torch.cuda.synchronize()
    assert torch.all(sc.sky == 0)
