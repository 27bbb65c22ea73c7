"""Pins of the oracle's scattering physics (Sec. 2.2, 3.5, 3.6) and sources (Sec. 3.2,
3.3): Henyey-Greenstein moments and CDF, normalisation of the peel-off phase
function, hand-computed Stokes cases of the White approximation, geometric facts
of the new direction, and the emission densities of point and sphere sources."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

EMPTY = dict(grid=S.homogeneous_grid(2, 0.0))


@pytest.mark.parametrize("g", [-0.6, -0.1, 0.0, 0.3, 0.5, 0.85])
def test_hg_sample_mean_cosine_is_g(g):
    from numpy.polynomial.legendre import leggauss

    x, w = leggauss(300)
    mu = np.array([O.hg_cos(g, 0.5 * (t + 1)) for t in x])
    assert 0.5 * np.sum(w * mu) == pytest.approx(g, abs=1e-10)


@pytest.mark.parametrize("g", [-0.5, 0.2, 0.7])
def test_hg_sample_inverts_the_cdf(g):
    # F(mu) = int_-1^mu (1-g^2) / (2 (1+g^2-2 g m)^1.5) dm, in closed form
    for v in np.linspace(0.0, 1.0, 41):
        mu = O.hg_cos(g, v)
        F = (1 - g * g) / (2 * g) * (1 / math.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
        assert F == pytest.approx(v, abs=1e-12)
    assert O.hg_cos(g, 0.0) == pytest.approx(-1.0, abs=1e-15)
    assert O.hg_cos(g, 1.0) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("g,p_l", [(0.0, 0.0), (0.5, 0.5), (-0.3, 1.0), (0.9, 0.2)])
def test_peel_phase_function_integrates_to_one_and_polarization_degree(g, p_l):
    """Peel-off of an unpolarized unit packet in an empty medium: I(mu) = P11/(4 pi)
    must integrate to one over the sphere of observer directions, and the degree of
    linear polarization must be p_l (1 - mu^2)/(1 + mu^2)."""
    from numpy.polynomial.legendre import leggauss

    x, w = leggauss(400 if g < 0.8 else 2000)
    total = 0.0
    for mu, wt in zip(x, w):
        th = math.acos(mu)
        prob = S.Problem(**EMPTY, g=g, p_l=p_l, theta_obs=th, phi_obs=0.3)
        ok, out = O.peel_packet(prob, [0.1, -0.2, 0.05], [0, 0, 1], [1, 0, 0], [1, 0, 0])
        assert ok
        total += wt * out[0] * 2 * math.pi
        pol = math.hypot(out[1], out[2]) / out[0]
        assert pol == pytest.approx(p_l * (1 - mu * mu) / (1 + mu * mu), abs=1e-12)
    assert total == pytest.approx(1.0, rel=1e-9)


def test_peel_of_polarized_light_at_right_angle():
    """Light along +z polarized along x (Q = 1 in the frame with reference x) seen by an
    observer on +x: the dipole axis points at the observer, so with p_l = 1, g = 0 the
    scattered intensity vanishes; an observer on +y sees it fully polarized with
    intensity doubled relative to unpolarized light (2 P11/(4 pi))."""
    P11 = 1.0  # g = 0
    prob = S.Problem(**EMPTY, g=0.0, p_l=1.0, theta_obs=math.pi / 2, phi_obs=0.0)
    ok, out = O.peel_packet(prob, [0, 0, 0], [0, 0, 1], [1, 0, 0], [1, 1, 0])
    assert ok and abs(out[0]) < 1e-15
    prob = S.Problem(**EMPTY, g=0.0, p_l=1.0, theta_obs=math.pi / 2, phi_obs=math.pi / 2)
    ok, out = O.peel_packet(prob, [0, 0, 0], [0, 0, 1], [1, 0, 0], [1, 1, 0])
    assert out[0] == pytest.approx(2 * P11 / (4 * math.pi), rel=1e-14)
    # E along x; the observer on +y has ex = (-1, 0, 0): horizontal on the sky -> Q = -I
    assert out[1] == pytest.approx(-out[0], rel=1e-14)
    assert abs(out[2]) < 1e-15


def test_peel_polarization_is_perpendicular_to_scattering_plane():
    """Unpolarized light from the origin scattered at pos: the polarization of the
    peeled packet is perpendicular to the plane (source, pos, observer), i.e.
    tangential on the sky: Q/I = P (x^2 - y^2)/r^2, U/I = P 2xy/r^2 (Q along the sky y
    axis, U toward 45 degrees between +y and -x)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        th, ph = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        prob = S.Problem(**EMPTY, g=0.3, p_l=0.7, theta_obs=th, phi_obs=ph)
        pos = rng.uniform(-1, 1, 3)
        n = pos / np.linalg.norm(pos)
        ref = np.cross(n, [0.3, 0.1, 1.0])
        ref /= np.linalg.norm(ref)
        ok, out = O.peel_packet(prob, pos, n, ref, [1, 0, 0])
        I, Q, U, x, y = out
        k = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        mu = float(n @ k)
        P = 0.7 * (1 - mu * mu) / (1 + mu * mu)
        r2 = x * x + y * y
        assert Q / I == pytest.approx(P * (x * x - y * y) / r2, abs=1e-10)
        assert U / I == pytest.approx(P * 2 * x * y / r2, abs=1e-10)
        # sky coordinates of the projection
        ex = np.array([-math.sin(ph), math.cos(ph), 0.0])
        ey = np.array([-math.cos(th) * math.cos(ph), -math.cos(th) * math.sin(ph), math.sin(th)])
        assert x == pytest.approx(pos @ ex, abs=1e-14) and y == pytest.approx(pos @ ey, abs=1e-14)


def test_peel_attenuation_by_medium():
    g = S.random_grid(4, seed=21)
    prob = S.Problem(grid=g, g=0.4, p_l=0.0, theta_obs=1.0, phi_obs=2.0)
    pos = np.array([0.2, -0.3, 0.1])
    n = np.array([0.0, 0.6, 0.8])
    ok, out = O.peel_packet(prob, pos, n, [1, 0, 0], [1, 0, 0])
    k = np.array([math.sin(1.0) * math.cos(2.0), math.sin(1.0) * math.sin(2.0), math.cos(1.0)])
    tau = O.tau_ray(prob, pos, k)
    mu = float(n @ k)
    hg = (1 - 0.16) / (1 + 0.16 - 0.8 * mu) ** 1.5
    assert out[0] == pytest.approx(math.exp(-tau) * hg / (4 * math.pi), rel=1e-13)


def test_scatter_geometry():
    """The new direction makes angle Theta(v) with the old one, its azimuth about the
    old direction measured from the reference axis is 2 pi u, and the new reference
    axis lies in the scattering plane, perpendicular to the new direction."""
    rng = np.random.default_rng(5)
    prob = S.Problem(**EMPTY, g=0.55, p_l=0.4)
    for _ in range(300):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        a = np.cross(n, rng.standard_normal(3))
        a /= np.linalg.norm(a)
        u, v = rng.uniform(), rng.uniform()
        n2, a2, _ = O.scatter_packet(prob, u, v, n, a, [1, 0, 0])
        assert np.linalg.norm(n2) == pytest.approx(1, abs=1e-14)
        assert n2 @ n == pytest.approx(O.hg_cos(0.55, v), abs=1e-12)
        b = np.cross(n, a)
        perp = n2 - (n2 @ n) * n
        if np.linalg.norm(perp) > 1e-6:
            perp /= np.linalg.norm(perp)
            ang = math.atan2(perp @ b, perp @ a) % (2 * math.pi)
            assert ang == pytest.approx(2 * math.pi * u, abs=1e-9) or abs(ang - 2 * math.pi * u) > 6.28
            m = np.cross(n, n2)
            m /= np.linalg.norm(m)
            assert abs(a2 @ n2) < 1e-12 and abs(a2 @ m) < 1e-12
            assert np.linalg.norm(a2) == pytest.approx(1, abs=1e-14)


def test_scatter_stokes_hand_cases():
    """Rayleigh-like dust (p_l = 1, g = 0) scattering light along +z polarized along the
    reference axis x by 90 degrees: in the plane of polarization (azimuth 0) the
    intensity vanishes; across it (azimuth 90 degrees) it doubles and the packet is
    fully polarized perpendicular to the new scattering plane."""
    prob = S.Problem(**EMPTY, g=0.0, p_l=1.0)
    n2, a2, S2 = O.scatter_packet(prob, 0.0, 0.5, [0, 0, 1], [1, 0, 0], [1, 1, 0])
    assert np.allclose(n2, [1, 0, 0], atol=1e-15)
    assert abs(S2[0]) < 1e-15
    n2, a2, S2 = O.scatter_packet(prob, 0.25, 0.5, [0, 0, 1], [1, 0, 0], [1, 1, 0])
    assert np.allclose(n2, [0, 1, 0], atol=1e-15)
    assert S2[0] == pytest.approx(2.0, abs=1e-14)
    assert S2[1] == pytest.approx(-2.0, abs=1e-14) and abs(S2[2]) < 1e-14
    # unpolarized dust (p_l = 0) keeps I and keeps an unpolarized packet unpolarized
    prob0 = S.Problem(**EMPTY, g=0.6, p_l=0.0)
    rng = np.random.default_rng(8)
    for _ in range(50):
        _, _, S3 = O.scatter_packet(prob0, rng.uniform(), rng.uniform(), [0, 0, 1], [1, 0, 0], [0.7, 0, 0])
        assert S3[0] == pytest.approx(0.7, rel=1e-15) and S3[1] == 0 and S3[2] == 0


def test_scatter_keeps_stokes_physical():
    rng = np.random.default_rng(10)
    prob = S.Problem(**EMPTY, g=0.4, p_l=0.8)
    for _ in range(500):
        p = rng.uniform(0, 1)
        chi = rng.uniform(0, math.pi)
        Sin = [1.0, p * math.cos(2 * chi), p * math.sin(2 * chi)]
        _, _, So = O.scatter_packet(prob, rng.uniform(), rng.uniform(), [0, 0, 1], [1, 0, 0], Sin)
        assert So[0] >= 0
        assert math.hypot(So[1], So[2]) <= So[0] * (1 + 1e-12) + 1e-15


def test_point_source_emission_is_eq_point_source_direction():
    prob = S.Problem(**EMPTY, generator="sobol")
    pts = O.generate_points("sobol", 3, 1, 64, "f64")
    for j in range(64):
        pos, d, e, w, depth = O.emit_packet(prob, j + 1)
        u, v, ww = pts[j]
        ref = [math.sqrt(1 - (2 * v - 1) ** 2) * math.cos(2 * math.pi * u),
               math.sqrt(1 - (2 * v - 1) ** 2) * math.sin(2 * math.pi * u), 2 * v - 1]
        assert np.allclose(d, ref, atol=1e-15) and np.allclose(pos, 0)
        assert depth == ww and w == 1.0
        assert abs(e @ d) < 1e-15


@pytest.mark.parametrize("order", ["direct", "inverse"])
def test_sphere_source_emission_density(order):
    """Emission points lie on the star, directions point outward, and the cosine of
    the emission angle has density 2 mu (isotropic surface), so E[mu] = 2/3; the limb
    darkening weight averages to one."""
    prob = S.Problem(**EMPTY, source="sphere", star_r=0.05, limb_u=0.6, emit_order=order,
                     generator="sobol")
    mus, ws = [], []
    for i in range(1, 4097):
        pos, d, e, w, depth = O.emit_packet(prob, i)
        assert np.linalg.norm(pos) == pytest.approx(0.05, rel=1e-12)
        mu = float(pos @ d) / 0.05
        assert mu >= -1e-12
        assert abs(e @ d) < 1e-12
        mus.append(mu)
        ws.append(w)
        assert w == pytest.approx((1 - 0.6 + 0.6 * mu) / (1 - 0.2), rel=1e-10)
    assert np.mean(mus) == pytest.approx(2 / 3, abs=2e-3)
    assert np.mean(ws) == pytest.approx(1.0, abs=2e-3)


def test_inverse_order_uses_point_source_direction_and_depth():
    """Inverse order: the first two coordinates give the direction exactly as for a
    point source and the third the depth (Sec. 3.3)."""
    ps = S.Problem(**EMPTY, generator="sobol")
    ss = S.Problem(**EMPTY, source="sphere", star_r=0.1, emit_order="inverse", generator="sobol")
    for i in range(1, 200):
        _, d0, _, _, w0 = O.emit_packet(ps.replace(source="point"), i)
        _, d1, _, _, w1 = O.emit_packet(ss, i)
        assert np.allclose(d0, d1, atol=1e-15) and w0 == w1


def test_occultation_by_the_star():
    prob = S.Problem(**EMPTY, source="sphere", star_r=0.1, theta_obs=math.pi / 2, phi_obs=0.0)
    ok, _ = O.peel_packet(prob, [-0.5, 0.0, 0.0], [1, 0, 0], [0, 0, 1], [1, 0, 0])
    assert not ok  # the star lies between the point and an observer on +x
    ok, _ = O.peel_packet(prob, [-0.5, 0.0, 0.2], [1, 0, 0], [0, 0, 1], [1, 0, 0])
    assert ok
    ok, _ = O.peel_packet(prob, [0.5, 0.0, 0.0], [1, 0, 0], [0, 0, 1], [1, 0, 0])
    assert ok


def test_quarter_turn_directions_are_exact():
    """phi = 2 pi u at u = 1/4, 1/2, 3/4 (Sobol indices 3, 1, 2) gives directions with an
    exactly zero x or y component, so rays from a source on a cell face stay on it."""
    prob = S.Problem(**EMPTY, generator="sobol")
    _, d1, _, _, _ = O.emit_packet(prob, 1)  # u = 1/2: phi = pi
    _, d2, _, _, _ = O.emit_packet(prob, 2)  # u = 3/4: phi = 3 pi / 2
    _, d3, _, _, _ = O.emit_packet(prob, 3)  # u = 1/4: phi = pi / 2
    assert d1[1] == 0.0 and d1[0] < 0
    assert d2[0] == 0.0 and d2[1] < 0
    assert d3[0] == 0.0 and d3[1] > 0
