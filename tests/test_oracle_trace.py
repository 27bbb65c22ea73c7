"""End-to-end pins of the oracle's tracer against closed forms, an independent
quadrature of the single-scattering integral, conservation of energy, independent
re-binning of the packet log, and limits the paper states (a small star acts as a
point source, Sec. 7)."""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S


def sphere_single_scattering_total(k, g=0.0, albedo=1.0, n=400):
    """Closed form of the scattered light from a point source at the centre of a
    homogeneous sphere (radius 1, extinction k), seen from any direction:
    (albedo/4 pi) int_0^1 k e^{-k r} (1/2) int_-1^1 e^{-k s(r,mu)} x_HG(mu) dmu dr,
    s(r, mu) = -r mu + sqrt(1 - r^2 (1 - mu^2)) the path to the surface."""
    x, w = leggauss(n)
    r, wr = 0.5 * (x + 1), 0.5 * w
    R, M = np.meshgrid(r, x, indexing="ij")
    s = -R * M + np.sqrt(1 - R ** 2 * (1 - M ** 2))
    hg = (1 - g * g) / (1 + g * g - 2 * g * M) ** 1.5
    inner = 0.5 * np.sum(w[None, :] * np.exp(-k * s) * hg, axis=1)
    return albedo * np.sum(wr * k * np.exp(-k * r) * inner) / (4 * math.pi)


@pytest.mark.parametrize("g,tol", [(0.0, 2e-6), (0.5, 2e-4), (-0.4, 2e-4)])
def test_homogeneous_sphere_total_matches_closed_form(g, tol):
    N = 1 << 16
    p = S.homogeneous_sphere_problem(g=g)
    img = O.trace_single(p, 1, N)
    assert img[0].sum() / N == pytest.approx(sphere_single_scattering_total(0.1, g), rel=tol)


def test_optically_thin_limit():
    k = 1e-4
    N = 1 << 14
    p = S.homogeneous_sphere_problem(sphere_k=k)
    tot = O.trace_single(p, 1, N)[0].sum() / N
    assert tot == pytest.approx(k / (4 * math.pi), rel=2e-4)


def test_sphere_integrated_polarization_vanishes():
    N = 1 << 16
    p = S.homogeneous_sphere_problem(g=0.4, p_l=0.5, sphere_k=1.0)
    img = O.trace_single(p, 1, N)
    I = img[0].sum()
    assert abs(img[1].sum()) < 2e-3 * I and abs(img[2].sum()) < 2e-3 * I
    # but the image itself is polarized (tangential pattern)
    assert np.abs(img[1]).sum() > 0.05 * I


def _bin_log(prob, log):
    img = np.zeros((3, prob.ny, prob.nx))
    ok = log[:, 8] == 0
    x, y, St = log[ok, 6], log[ok, 7], log[ok, 3:6]
    fx = (x + prob.half_width) / (2 * prob.half_width) * prob.nx
    fy = (y + prob.half_width) / (2 * prob.half_width) * prob.ny
    if prob.splat == "nearest":
        ix, iy = np.floor(fx).astype(int), np.floor(fy).astype(int)
        inside = (ix >= 0) & (ix < prob.nx) & (iy >= 0) & (iy < prob.ny)
        for s in range(3):
            np.add.at(img[s], (iy[inside], ix[inside]), St[inside, s])
        return img
    fx, fy = fx - 0.5, fy - 0.5
    x0, y0 = np.floor(fx), np.floor(fy)
    ax, ay = fx - x0, fy - y0
    for dy in (0, 1):
        for dx in (0, 1):
            ix, iy = (x0 + dx).astype(int), (y0 + dy).astype(int)
            wgt = (ax if dx else 1 - ax) * (ay if dy else 1 - ay)
            inside = (ix >= 0) & (ix < prob.nx) & (iy >= 0) & (iy < prob.ny)
            for s in range(3):
                np.add.at(img[s], (iy[inside], ix[inside]), (wgt * St[:, s])[inside])
    return img


@pytest.mark.parametrize("splat", ["nearest", "bilinear"])
def test_image_is_the_binned_packet_log(splat):
    p = S.flared_disk_problem(n=32, nx=48, ny=40, half_width=0.9, splat=splat)
    img, log = O.trace_single(p, 1, 1 << 12, log=True)
    assert np.allclose(img, _bin_log(p, log), rtol=1e-12, atol=1e-16)


def test_packet_log_follows_forced_scattering_and_peel_off():
    """Per packet: the scattering point lies on the emission ray at optical depth
    -ln[1 - w(1 - e^{-tau_1})] (Eq. random_depth), and the peel-off intensity is
    albedo (1 - e^{-tau_1}) e^{-tau_obs} x_HG / (4 pi); every optical depth here is
    recomputed by a fine midpoint rule, not by the oracle's cell walk."""
    grid = S.random_grid(3, seed=2, kmax=1.5)
    p = S.Problem(grid=grid, albedo=0.8, g=0.3, p_l=0.4, theta_obs=1.1, phi_obs=0.7, half_width=1.5)
    N = 96
    _, log = O.trace_single(p, 1, N, log=True)
    pts = O.generate_points("sobol", 3, 1, N, "f64")
    k = np.array([math.sin(1.1) * math.cos(0.7), math.sin(1.1) * math.sin(0.7), math.cos(1.1)])

    def mid_tau(p0, d, t_end, steps=200_000):
        t = (np.arange(steps) + 0.5) * (t_end / steps)
        x = p0[None, :] + t[:, None] * d[None, :]
        idx = np.clip(np.floor((x + 1) / 2 * 3).astype(int), 0, 2)
        return grid[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64).sum() * (t_end / steps)

    def exit_t(p0, d):
        return min(((1 if d[a] > 0 else -1) - p0[a]) / d[a] for a in range(3) if d[a] != 0)

    for j in range(N):
        u, v, w = pts[j]
        ct = 2 * v - 1
        d = np.array([math.sqrt(1 - ct * ct) * math.cos(2 * math.pi * u),
                      math.sqrt(1 - ct * ct) * math.sin(2 * math.pi * u), ct])
        pos = log[j, 0:3]
        t = float(pos @ d)
        assert np.allclose(pos, t * d, atol=1e-12)
        tau1 = mid_tau(np.zeros(3), d, exit_t(np.zeros(3), d))
        W1 = 1 - math.exp(-tau1)
        assert mid_tau(np.zeros(3), d, t) == pytest.approx(-math.log(1 - w * W1), rel=1e-3, abs=1e-6)
        tau_obs = mid_tau(pos, k, exit_t(pos, k))
        mu = float(d @ k)
        hg = (1 - 0.09) / (1 + 0.09 - 0.6 * mu) ** 1.5
        assert log[j, 3] == pytest.approx(0.8 * W1 * math.exp(-tau_obs) * hg / (4 * math.pi), rel=2e-3)


def test_single_scattering_matches_independent_quadrature_on_tiny_grid():
    """The scattered light of a point source in a tiny random grid, observed along +x,
    written as the physical integral over emission directions and path length:
    (albedo/4pi) int dOmega/(4pi) int_0^s k(t) e^{-tau(0,t)} e^{-tau_obs(t)} x_HG dt.
    Directions by Gauss-Legendre in cos(theta) x midpoint in phi; the path by a fine
    midpoint rule with cumulative sums; tau_obs from exact row sums along +x."""
    n = 3
    grid = S.random_grid(n, seed=17, kmax=1.2).astype(np.float64)
    albedo, g = 0.8, 0.35
    h = 2.0 / n
    # tau from a point to the +x face: partial cell + whole cells beyond
    tail = np.concatenate([np.cumsum(grid[:, :, ::-1], axis=2)[:, :, ::-1][:, :, 1:] * h,
                           np.zeros((n, n, 1))], axis=2)
    xm, wm = leggauss(96)
    nphi, nt = 192, 1500
    total = 0.0
    for mu, wmu in zip(xm, wm):
        st = math.sqrt(1 - mu * mu)
        phi = (np.arange(nphi) + 0.5) * (2 * math.pi / nphi)
        d = np.stack([st * np.cos(phi), st * np.sin(phi), np.full(nphi, mu)], axis=1)
        with np.errstate(divide="ignore"):
            tex = np.min(np.where(d != 0, (np.sign(d) - 0.0) / np.where(d != 0, d, 1), np.inf), axis=1)
        for q in range(nphi):
            dt = tex[q] / nt
            t = (np.arange(nt) + 0.5) * dt
            x = t[:, None] * d[q][None, :]
            c = np.clip(np.floor((x + 1) / h).astype(int), 0, n - 1)
            kc = grid[c[:, 2], c[:, 1], c[:, 0]]
            tau = np.cumsum(kc) * dt - 0.5 * kc * dt
            xr = -1 + (c[:, 0] + 1) * h
            tobs = (xr - x[:, 0]) * kc + tail[c[:, 2], c[:, 1], c[:, 0]]
            mu_o = d[q][0]
            hg = (1 - g * g) / (1 + g * g - 2 * g * mu_o) ** 1.5
            total += wmu / 2 / nphi * np.sum(kc * np.exp(-tau - tobs)) * dt * hg
    ref = albedo * total / (4 * math.pi)
    p = S.Problem(grid=grid.astype(np.float32), albedo=albedo, g=g, theta_obs=math.pi / 2, phi_obs=0.0,
                  half_width=1.8, nx=16, ny=16)
    N = 1 << 18
    got = O.trace_single(p, 1, N)[0].sum() / N
    assert got == pytest.approx(ref, rel=2e-3)


def test_multiple_scattering_first_order_equals_single():
    """Coordinates 0, 1, 2 of order 1 are the single-scattering coordinates, so the
    order-1 image of the multiple-scattering tracer is the single-scattering image."""
    p = S.clumpy_problem(n=32, max_orders=5, nx=64, ny=64, per_order=True)
    multi = O.trace_multiple(p, 1, 1 << 12)
    single = O.trace_single(p.replace(max_orders=1, per_order=False), 1, 1 << 12)
    assert np.array_equal(multi[0], single)
    assert multi[1:].sum() > 0


def test_energy_conservation_homogeneous_sphere():
    """Albedo 1, isotropic scattering, every order forced, no roulette: the peel-off
    light summed over all orders and integrated over all observer directions equals
    the light that scatters at least once, 1 - e^{-k} for a central source.  By
    symmetry the integral is 4 pi times the image total seen from one direction."""
    k = 0.6
    p = S.homogeneous_sphere_problem(sphere_k=k, max_orders=30, albedo=1.0, g=0.0, generator="sobol")
    N = 1 << 14
    tot = 0.0
    dirs = [(math.pi / 2, 0.0), (0.3, 1.0), (2.2, 4.0), (1.0, 2.5)]
    for th, ph in dirs:
        img = O.trace_multiple(p.replace(theta_obs=th, phi_obs=ph), 1, N)
        tot += 4 * math.pi * img[:, 0].sum() / N / len(dirs)
    assert tot == pytest.approx(1 - math.exp(-k), rel=3e-3)


def test_energy_conservation_with_albedo_and_unforced_orders():
    """With albedo w and isotropic scattering in a sphere the escaping scattered light
    is the same for every forcing variant; forcing only the first order (the paper's
    variant) and forcing all orders must agree within sampling error, and both stay
    below 1 - e^{-k}."""
    k = 0.8
    base = S.homogeneous_sphere_problem(sphere_k=k, max_orders=25, albedo=0.9, g=0.2, generator="sobol_owen",
                                        seed=5)
    N = 1 << 15
    a = O.trace_multiple(base, 1, N)[:, 0].sum() / N
    b = O.trace_multiple(base.replace(force="first"), 1, N)[:, 0].sum() / N
    assert a == pytest.approx(b, rel=1e-2)
    assert 4 * math.pi * a < 1 - math.exp(-k)


def test_roulette_is_unbiased():
    p = S.clumpy_problem(n=32, max_orders=12, nx=32, ny=32, rr_threshold=0.0)
    N = 1 << 13
    ref = O.trace_multiple(p, 1, N)[0, 0].sum()
    rr = O.trace_multiple(p.replace(rr_threshold=0.05, rr_survival=0.3), 1, N)[0, 0].sum()
    assert rr == pytest.approx(ref, rel=3e-2)
    assert rr != ref


def test_small_star_inverse_order_is_the_point_source():
    """Inverse order uses the point-source coordinates for direction and depth, so a
    star of vanishing radius (no limb darkening) gives the point-source image."""
    p = S.flared_disk_problem(n=32, nx=64, ny=64)
    N = 1 << 13
    pt = O.trace_single(p, 1, N)
    st = O.trace_single(p.replace(source="sphere", star_r=1e-9, emit_order="inverse"), 1, N)
    assert np.abs(st - pt).sum() <= 1e-6 * np.abs(pt).sum()


def test_direct_and_inverse_order_agree_statistically():
    """Both number orders estimate the same integral: totals agree and the image-based
    norm of Eq. norm between them shrinks as the point count grows."""
    p = S.flared_disk_problem(n=32, nx=16, ny=16, source="sphere", star_r=0.05, limb_u=0.6)
    norms = []
    for N in (1 << 14, 1 << 18):
        a = O.trace_single(p.replace(emit_order="direct"), 1, N)[0]
        b = O.trace_single(p.replace(emit_order="inverse"), 1, N)[0]
        assert a.sum() == pytest.approx(b.sum(), rel=5e-3)
        norms.append(np.abs(a - b).sum() / (np.abs(a + b).sum() / 2))
    assert norms[1] < 0.05 and norms[1] < 0.4 * norms[0]


def test_hammersley_last_point_is_valid():
    p = S.flared_disk_problem(n=16, nx=16, ny=16, generator="hammersley", total_n=1000)
    img = O.trace_single(p, 1, 1000)
    assert np.all(np.isfinite(img))


def test_three_d_reuse_anti_pattern_does_not_converge():
    """Reusing one 3-D point per order (Sec. 6 warns against it) correlates the orders:
    the second-order image then disagrees with the long-vector estimate by far more
    than the sampling error, and the gap does not shrink with N."""
    p = S.homogeneous_sphere_problem(sphere_k=1.0, max_orders=2, per_order=True, g=0.3, generator="sobol")

    def reuse_second_order(N):
        # the 12-D vector of an order-2 packet filled with the same 3 coordinates twice
        pts = O.generate_points("sobol", 3, 1, N, "f64")
        from oracle.oracle import _Holder  # noqa: F401  (only to keep the oracle loaded)

        tot = 0.0
        for (u, v, w) in pts:
            # order 1: direction and depth
            ct = 2 * v - 1
            n = np.array([math.sqrt(1 - ct * ct) * math.cos(2 * math.pi * u),
                          math.sqrt(1 - ct * ct) * math.sin(2 * math.pi * u), ct])
            s = 1.0
            W1 = 1 - math.exp(-s)
            r = -math.log(1 - w * W1)
            pos = r * n
            a = np.cross(n, [0.0, 0.0, 1.0]) if abs(ct) < 0.99 else np.array([1.0, 0.0, 0.0])
            a /= np.linalg.norm(a)
            n2, a2, S2 = O.scatter_packet(p, u, v, n, a, [W1, 0, 0])
            hit_t = O.tau_ray(p, pos, n2)
            W2 = 1 - math.exp(-hit_t)
            ok, q = O.march_ray(p, pos, n2, -math.log(1 - w * W2))
            ok, out = O.peel_packet(p, q, n2, a2, [S2[0] * W2, 0, 0])
            tot += out[0]
        return tot / N

    good = O.trace_multiple(p, 1, 1 << 14)[1, 0].sum() / (1 << 14)
    bad_small, bad_large = reuse_second_order(1 << 10), reuse_second_order(1 << 12)
    assert abs(bad_large - good) > 0.02 * good
    assert abs(bad_large - good) > 0.5 * abs(bad_small - good)


def test_identity_warp_is_the_plain_tracer_and_logs_packet_totals():
    """x = u with log J = 0 replays the plain multiple-scattering tracer exactly; the
    training log holds the point's first coordinates, its per-packet sums of in-image
    intensity add up to the image total, and its per-packet L2 norms lie between
    sum / sqrt(orders) and the sum."""
    p = S.clumpy_problem(n=16, max_orders=6, nx=32, ny=32, half_width=0.6)
    N = 1 << 12
    u = O.generate_points("sobol", 3, 1, N)
    plain = O.trace_multiple(p, 1, N)
    img, log = O.trace_multiple_warped(p, 1, N, u, np.zeros(N), train_log=True)
    assert np.array_equal(img, plain)
    img2, log2 = O.trace_multiple_warped(p, 1, N, train_log=True)
    assert np.array_equal(img2, plain) and np.array_equal(log2, log)
    assert np.array_equal(log[:, :3], u)
    assert np.all(log[:, 3] >= 0)
    assert log[:, 3].sum() == pytest.approx(img[0, 0].sum(), rel=1e-12)
    assert np.all(log[:, 4] <= log[:, 3] * (1 + 1e-12))
    assert np.all(log[:, 4] >= log[:, 3] / np.sqrt(p.max_orders) * (1 - 1e-12))
    assert np.any(log[:, 4] < log[:, 3] * (1 - 1e-3))


@pytest.mark.parametrize("use_jacobian", [True, False])
def test_warped_estimator_keeps_energy_conservation(use_jacobian):
    """A known bijection of the first-order coordinates (x1 = u1^2, x2 = u2^3, with
    |dx/du| = 2 u1 * 3 u2^2) leaves the homogeneous-sphere energy balance
    1 - e^{-k} intact when the weight carries the Jacobian, and breaks it when the
    Jacobian is dropped."""
    k = 0.6
    p = S.homogeneous_sphere_problem(sphere_k=k, max_orders=30, albedo=1.0, g=0.0, generator="sobol")
    N = 1 << 14
    u = O.generate_points("sobol", 3, 1, N)
    x = u.copy()
    x[:, 1] = u[:, 1] ** 2
    x[:, 2] = u[:, 2] ** 3
    logj = np.log(2 * u[:, 1]) + np.log(3 * u[:, 2] ** 2) if use_jacobian else np.zeros(N)
    tot = 0.0
    dirs = [(math.pi / 2, 0.0), (0.3, 1.0), (2.2, 4.0), (1.0, 2.5)]
    for th, ph in dirs:
        img = O.trace_multiple_warped(p.replace(theta_obs=th, phi_obs=ph), 1, N, x, logj)
        tot += 4 * math.pi * img[:, 0].sum() / N / len(dirs)
    err = abs(tot / (1 - math.exp(-k)) - 1)
    if use_jacobian:
        assert err < 2e-3
    else:
        assert err > 5e-3


def test_direct_light_of_a_point_source_in_a_homogeneous_sphere():
    """e^-kR / (4 pi) in the pixel holding the sky origin, nothing elsewhere."""
    k = 0.7
    p = S.homogeneous_sphere_problem(sphere_k=k, nx=9, ny=9)
    img = O.direct_light(p)
    assert img[0, 4, 4] == pytest.approx(math.exp(-k) / (4 * math.pi), rel=1e-14)
    assert img[0].sum() == pytest.approx(img[0, 4, 4], rel=1e-14) and np.all(img[1:] == 0)


@pytest.mark.parametrize("u", [0.0, 0.6, 1.0])
def test_direct_light_of_a_star_in_vacuum_integrates_to_one_over_4pi(u):
    """Surface brightness normalised so the disk holds 1 / (4 pi): the midpoint-rule
    total converges to it as the subsampling grows; for a uniform disk (u = 0) a
    pixel the disk covers completely holds exactly its area share."""
    p = S.Problem(grid=np.zeros((4, 4, 4), np.float32), source="sphere", star_r=0.5, limb_u=u, theta_obs=0.9,
                  phi_obs=0.4, half_width=0.6, nx=24, ny=24)
    totals = [O.direct_light(p, s)[0].sum() for s in (2, 8, 32)]
    errs = [abs(t * 4 * math.pi - 1) for t in totals]
    assert errs[2] < 2e-3 and errs[2] < errs[0]
    if u == 0.0:
        img = O.direct_light(p, 3)[0]
        pix = (2 * 0.6 / 24) ** 2
        assert img[12, 12] == pytest.approx(pix / (math.pi * 0.25) / (4 * math.pi), rel=1e-12)


def test_direct_light_of_a_star_is_dimmed_by_the_medium_in_front():
    """A slab of extinction in front of the star (toward the observer) dims every
    pixel by e^-(k L) with L the slab thickness along the line of sight, when the slab
    is crossed completely; an empty grid changes nothing."""
    n = 8
    grid = np.zeros((n, n, n), np.float32)
    grid[:, :, 6] = 2.0  # x in [0.5, 0.75): a slab across the x axis, in front of an observer on +x
    base = S.Problem(grid=np.zeros((n, n, n), np.float32), source="sphere", star_r=0.3, limb_u=0.5,
                     theta_obs=math.pi / 2, phi_obs=0.0, half_width=0.4, nx=16, ny=16)
    clear = O.direct_light(base, 4)[0]
    dim = O.direct_light(base.replace(grid=grid), 4)[0]
    mask = clear > 0
    assert np.allclose(dim[mask] / clear[mask], math.exp(-2.0 * 0.25), rtol=1e-12)


def test_multiple_scattering_from_a_vanishing_star_is_the_point_source():
    """Inverse order reads direction and first depth from coordinates 0, 1, 2 as the
    point source does (its two emission coordinates come after all orders'), so a star
    of vanishing radius gives the point-source image of multiple scattering.  (Owen-
    scrambled points: unscrambled Sobol points send some rays exactly along the cell
    faces through the origin, where a source 1e-9 off the face sees the neighbouring
    column of cells.)"""
    p = S.clumpy_problem(n=16, max_orders=5, nx=32, ny=32, generator="sobol_owen", seed=5)
    N = 1 << 12
    pt = O.trace_multiple(p, 1, N)
    st = O.trace_multiple(p.replace(source="sphere", star_r=1e-9, emit_order="inverse"), 1, N)
    assert np.abs(st - pt).sum() <= 1e-6 * np.abs(pt).sum()


@pytest.mark.parametrize("order", ["inverse", "direct"])
def test_energy_conservation_of_a_small_star(order):
    """A star of radius 1e-3 (uniform disk) at the centre of the homogeneous sphere:
    with albedo 1 and every order forced the scattered light integrated over all
    directions is 1 - e^-k(1 - R) up to the star's own size."""
    k = 0.6
    p = S.homogeneous_sphere_problem(sphere_k=k, max_orders=30, albedo=1.0, g=0.0, source="sphere", star_r=1e-3,
                                     limb_u=0.0, emit_order=order)
    N = 1 << 14
    tot = 0.0
    dirs = [(math.pi / 2, 0.0), (0.3, 1.0), (2.2, 4.0), (1.0, 2.5)]
    for th, ph in dirs:
        img = O.trace_multiple(p.replace(theta_obs=th, phi_obs=ph), 1, N)
        tot += 4 * math.pi * img[:, 0].sum() / N / len(dirs)
    assert tot == pytest.approx(1 - math.exp(-k), rel=4e-3)
