"""The tail map of an observer direction (qmcrt_tail_map): its code for a cell bounds the
optical depth the oracle integrates from any point of that cell along the direction to the
edge of the grid, and a trace whose peel-off walks stop on it changes each contribution by
at most the tolerance it was given."""
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


def _uneven():
    """A box of unequal sides with cells of unequal edges (11 x 6 x 9 cells), sparse."""
    rng = np.random.default_rng(21)
    g = rng.uniform(0.0, 3.0, size=(9, 6, 11)) * (rng.uniform(size=(9, 6, 11)) > 0.6)
    return S.Problem(grid=g.astype(np.float32), lo=(-1.0, -0.4, -2.0), hi=(1.5, 0.8, 0.7))


def _blobs():
    """Dense boxes in an empty box of unequal cells (15 x 12 x 13): the bound is tight, so a
    block a walk can reach but the map leaves out shows."""
    rng = np.random.default_rng(5)
    g = np.zeros((13, 12, 15), dtype=np.float32)
    for _ in range(8):
        size = rng.integers(2, 7, size=3)
        at = rng.integers(0, np.array(g.shape) - size + 1)
        g[at[0]:at[0] + size[0], at[1]:at[1] + size[1], at[2]:at[2] + size[2]] = rng.uniform(0.5, 4.0)
    return S.Problem(grid=g, lo=(-1.2, -0.9, -1.0), hi=(1.0, 1.1, 0.8))


MEDIA = {
    "disk": S.flared_disk_problem(n=32, nx=16, ny=16),
    "blobs": _blobs(),
    "fractal": S.fractal_cloud_problem(n=24, nx=16, ny=16),
    "clumpy": S.clumpy_problem(n=16, max_orders=1, nx=16, ny=16),
    "uneven": _uneven(),
}

DIRECTIONS = [(math.pi / 4, 0.0), (0.0, 0.0), (math.pi / 2, 0.0), (math.pi / 2, math.pi / 2), (1.1, 2.3),
              (2.0, 4.0), (math.pi, 0.0), (0.3, -0.7)]


def _k(theta, phi):
    return np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])


def _codes(Q, sc):
    """The map as a [nz][ny][nx] array of the grid proper's cells."""
    nz, ny, nx = sc.grid.shape
    p = sc.pad
    m = sc.tail.cpu().numpy().reshape(nz + 2 * p, ny + 2 * p, nx + 2 * p)
    return m, m[p:p + nz, p:p + ny, p:p + nx]


@pytest.mark.parametrize("theta,phi", DIRECTIONS)
@pytest.mark.parametrize("name", list(MEDIA))
def test_map_bounds_the_oracle_depth_from_every_point(Q, name, theta, phi):
    import torch

    prob = MEDIA[name].replace(theta_obs=theta, phi_obs=phi)
    sc = Q.Scene(prob, tail=True)
    torch.cuda.synchronize()
    full, codes = _codes(Q, sc)
    p = sc.pad
    assert not full[:p].any() and not full[-p:].any() and not full[:, :p].any() and not full[:, :, -p:].any()
    nz, ny, nx = codes.shape
    lo, hi = np.array(prob.lo), np.array(prob.hi)
    h = (hi - lo) / np.array([nx, ny, nz])
    k = _k(theta, phi)
    raw = prob.replace(kscale=1.0)
    rng = np.random.default_rng(7)
    # points anywhere in the box, and points just inside cell corners (the worst starts)
    pts = list(lo + rng.uniform(size=(600, 3)) * (hi - lo))
    for _ in range(200):
        c = rng.integers(0, [nx, ny, nz])
        pts.append(lo + (c + np.where(rng.integers(0, 2, size=3) == 1, 1 - 1e-6, 1e-6)) * h)
    checked = 0
    for q in pts:
        c = np.minimum(np.floor((q - lo) / h).astype(int), [nx - 1, ny - 1, nz - 1])
        code = int(codes[c[2], c[1], c[0]])
        tau = O.tau_ray(raw, q, k)
        if code == 0:
            assert tau == 0.0, (q, tau)
        elif code < 255:
            assert tau <= 2.0 ** (code - 150), (q, tau, code)
            checked += 1
    assert checked > 0 or not codes.any()


def _log(Q, prob, first, count, precision, tail):
    import torch

    sc = Q.Scene(prob, tail=tail)
    lg = torch.zeros((count, 9), dtype=torch.float64, device="cuda")
    buf = sc.accum_buffer("f64")
    sc.trace(first, count, buf, accum="f64", precision=precision, log=lg)
    torch.cuda.synchronize()
    return lg.cpu().numpy()


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("name", ["disk", "fractal", "clumpy"])
def test_each_contribution_changes_by_at_most_the_tolerance(Q, name, precision):
    """Per packet: the same scattering point, sky position and status, and I, Q, U within
    the tolerance (relative: e^{-tau_obs} grows by at most e^eps - 1)."""
    prob = MEDIA[name].replace(theta_obs=1.0, phi_obs=0.4)
    N = 1 << 14
    a = _log(Q, prob, 1, N, precision, True)
    b = _log(Q, prob, 1, N, precision, False)
    assert np.array_equal(a[:, [0, 1, 2, 6, 7, 8]], b[:, [0, 1, 2, 6, 7, 8]])
    eps = Q.TAIL_EPS[precision]
    ulp = 2.0 ** -23 if precision == "f32" else 2.0 ** -52  # the roundings of two traces
    ok = b[:, 8] == 0
    assert ok.sum() > N // 4
    I = np.abs(b[ok, 3])
    for c in (3, 4, 5):
        assert np.all(np.abs(a[ok, c] - b[ok, c]) <= (1.01 * eps + 8 * ulp) * I), c
    assert np.all(a[ok, 3] >= b[ok, 3] * (1 - 8 * ulp))  # depths left out only raise e^{-tau_obs}


def test_without_a_tolerance_the_map_leaves_out_only_empty_cells(Q):
    """tail_eps = 0 stops only where the map bounds what is left by zero (the empty
    corners of the envelope's box): each contribution agrees to within the rounding of
    the compensated sum, in FP64."""
    import torch

    prob = MEDIA["clumpy"].replace(theta_obs=0.7, phi_obs=2.0)
    logs = []
    for tail in (True, False):
        sc = Q.Scene(prob, tail=tail)
        lg = torch.zeros((1 << 14, 9), dtype=torch.float64, device="cuda")
        buf = sc.accum_buffer("f64")
        pts = Q.points_desc(prob.generator, prob.dims, 1, 1 << 14)
        opts = sc.opts("f64")
        opts.tail_eps = 0.0
        Q.qmcrt_trace_single(sc.medium, sc.source, sc.dust, sc.obs, pts, opts, sc.image_desc(buf, "f64"),
                             lg.data_ptr(), 0)
        torch.cuda.synchronize()
        logs.append(lg.cpu().numpy())
    a, b = logs
    assert np.array_equal(a[:, [0, 1, 2, 6, 7, 8]], b[:, [0, 1, 2, 6, 7, 8]])
    assert np.all(np.abs(a[:, 3:6] - b[:, 3:6]) <= 1e-14 * np.abs(b[:, 3:4]))


def test_batch_maps_follow_a_new_grid(Q):
    """A batch keeps the addresses of its instances' tail maps: after the scene's grid
    changes, repad rebuilds them in place and the batch still equals lone traces of the
    new grid bit for bit."""
    import torch

    prob = S.finite_star_disk_problem(n=32, nx=40, ny=36)
    inst = [S.Instance(theta_obs=th, albedo=0.6, g=0.4, kscale=ks, n_packets=2048, first_index=2048)
            for th, ks in ((0.3, 1.0), (1.2, 2.0), (2.5, 0.7))]
    sc = Q.Scene(prob)
    B = Q.Batch(prob, inst, scene=sc, chunk_log2=10, frac_bits=40)
    B.run()
    sc.grid.mul_(3.0)
    sc.repad()
    B.run()
    torch.cuda.synchronize()
    got = B.accum.cpu().numpy()
    for k, I in enumerate(inst):
        p = prob.replace(grid=prob.grid * 3.0, theta_obs=I.theta_obs, albedo=I.albedo, g=I.g, kscale=I.kscale)
        lone = Q.Scene(p)
        buf = lone.accum_buffer("i64")
        lone.trace(I.first_index, I.n_packets, buf, frac_bits=40)
        torch.cuda.synchronize()
        assert np.array_equal(got[k], buf[0, 0].cpu().numpy()), k
