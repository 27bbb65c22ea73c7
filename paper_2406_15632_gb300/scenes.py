"""Seeded synthetic inputs: problem descriptions and density grids.

This module holds no step of the radiative-transfer method.  It only describes
problems (medium, source, dust, observer, point set, trace options) and fills
density grids from closed-form density laws, so that the CUDA path and the CPU
oracle receive identical inputs.  Random numbers drawn here (the clump field, the
packet budgets of the batched workload) are scene inputs, not numbers the method
draws.

Geometries follow the shapes of the paper's tests (Sec. 5): a flared disk
(Eq. flared_disk), a spherical envelope (Eq. sphere) and a clumpy cloud standing in
for the fractal cloud, with sizes from the workloads this library is measured on.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

GENERATORS = ("sobol", "sobol_owen", "halton", "hammersley", "philox", "niederreiter", "faure")


@dataclass
class Problem:
    """One tracing problem.  Angles in radians; lengths in units of the medium."""

    # medium: a Cartesian grid of extinction per unit length (kappa * rho), cells
    # constant, x fastest ([nz, ny, nx]); or, when grid is None, a homogeneous
    # sphere of radius sphere_r and extinction sphere_k centred at the origin.
    grid: np.ndarray | None = None
    lo: tuple = (-1.0, -1.0, -1.0)
    hi: tuple = (1.0, 1.0, 1.0)
    kscale: float = 1.0
    sphere_r: float = 1.0
    sphere_k: float = 0.0
    # source at the origin: "point" or "sphere" (radius star_r, linear limb
    # darkening limb_u, number order "direct" or "inverse")
    source: str = "point"
    star_r: float = 0.0
    limb_u: float = 0.0
    emit_order: str = "inverse"
    # dust
    albedo: float = 1.0
    g: float = 0.0
    p_l: float = 0.0
    # observer and image: [3][ny][nx] Stokes I, Q, U over [-hw, hw]^2
    theta_obs: float = 0.0
    phi_obs: float = 0.0
    half_width: float = 1.0
    nx: int = 64
    ny: int = 64
    splat: str = "nearest"  # or "bilinear"
    # point set
    generator: str = "sobol"
    seed: int = 0
    total_n: int = 0  # N of the Hammersley set
    # trace options
    tau_min: float = 1e-12
    max_orders: int = 1
    rr_threshold: float = 0.0
    rr_survival: float = 0.1
    force: str = "all"  # "all" orders forced, or "first" only
    per_order: bool = False

    @property
    def dims(self) -> int:
        """Coordinates one packet consumes (one long vector per packet, Sec. 3.7)."""
        if self.max_orders > 1:  # a finite star's two extra emission coordinates go last
            return 4 * self.max_orders + (2 if self.source == "sphere" else 0)
        return 5 if self.source == "sphere" else 3

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    @property
    def n_images(self) -> int:
        return self.max_orders if (self.per_order and self.max_orders > 1) else 1


def cell_centres(n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def flared_disk_grid(n: int = 256, k0: float = 1.0 / 9.0, r_in: float = 0.1, r_out: float = 1.0,
                     h0: float = 0.1, beta: float = 1.25, alpha: float = 2.0) -> np.ndarray:
    """kappa*rho = k0 r^-alpha exp(-z^2 / 2 h^2), h = h0 r^beta, r_in <= r <= r_out
    (cylindrical r), sampled at cell centres of [-1, 1]^3.  With alpha = 2 and
    k0 = 1/9 the midplane optical depth from r_in = 0.1 to r_out = 1 is 1."""
    c = cell_centres(n)
    z = c[:, None, None]
    y = c[None, :, None]
    x = c[None, None, :]
    r = np.sqrt(x * x + y * y)
    rr = np.where(r > 0, r, 1.0)
    h = h0 * rr ** beta
    k = k0 * rr ** (-alpha) * np.exp(-0.5 * (z / h) ** 2)
    k = np.where((r >= r_in) & (r <= r_out), k, 0.0)
    return np.ascontiguousarray(k.astype(np.float32))


def homogeneous_grid(n: int = 4, k: float = 1.0) -> np.ndarray:
    return np.full((n, n, n), k, dtype=np.float32)


def random_grid(n: int = 4, seed: int = 0, kmax: float = 2.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, kmax, size=(n, n, n)).astype(np.float32)


def shell_envelope_grid(n: int = 256, r_in: float = 500.0 / 600.0, r_out: float = 550.0 / 600.0,
                        tau: float = 0.1) -> np.ndarray:
    """The paper's dust sphere envelope (Eq. sphere): constant density between r_in and
    r_out (500 and 550 au on a 600 au half-width cube), sampled at cell centres of
    [-1, 1]^3; the radial optical depth of the shell is tau (the paper gives the
    density in g cm^-3 without the opacity, so the depth is a chosen value)."""
    c = cell_centres(n)
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    k = np.where((r >= r_in) & (r <= r_out), tau / (r_out - r_in), 0.0)
    return np.ascontiguousarray(k.astype(np.float32))


def clumpy_envelope_grid(n: int = 128, tau_radial: float = 5.0, r_in: float = 0.05, r_out: float = 1.0,
                         power: float = 1.5, sigma: float = 1.0, corr_cells: float = 4.0,
                         seed: int = 20240622) -> np.ndarray:
    """Envelope kappa*rho = k0 r^-power (r_in <= r <= r_out) times a log-normal clump
    factor exp(sigma G - sigma^2/2), G a unit-variance Gaussian field: seeded white
    noise smoothed by a Gaussian of corr_cells cells (periodic FFT convolution).  k0
    is set analytically so that the smooth envelope's radial optical depth from the
    centre to r_out is tau_radial; the clump factor has mean one."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    f = np.fft.fftfreq(n)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    kern = np.exp(-2.0 * (math.pi * corr_cells) ** 2 * (kx * kx + ky * ky + kz * kz))
    G = np.real(np.fft.ifftn(np.fft.fftn(white) * kern))
    G = (G - G.mean()) / G.std()
    c = cell_centres(n)
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    integral = (r_out ** (1 - power) - r_in ** (1 - power)) / (1 - power)
    k0 = tau_radial / integral
    rr = np.where(r > 0, r, 1.0)
    k = k0 * rr ** (-power) * np.exp(sigma * G - 0.5 * sigma * sigma)
    k = np.where((r >= r_in) & (r <= r_out), k, 0.0)
    return np.ascontiguousarray(k.astype(np.float32))


def fractal_cloud_points(N: int = 32, D: float = 2.3, levels: int = 4, seed: int = 1556) -> np.ndarray:
    """Hierarchically clumped points in the unit cube [0, 1)^3 (Elmegreen 1997; Mathis
    et al. 2002; the paper's fractal cloud, Sec. 5): N uniform points in the cube; around
    each point a cube of edge 1 / (2 N^(1/D)) times the parent's edge, centred on it,
    receives N uniform points; repeated until `levels` generations (N^levels points);
    coordinates outside the unit cube are wrapped by one cube length.  The paper draws
    its points from L'Ecuyer's generator with seed -1556; here a seeded Philox stream
    of NumPy supplies the uniform triples."""
    rng = np.random.Generator(np.random.Philox(seed))
    pts = rng.uniform(0.0, 1.0, size=(N, 3))
    edge = 1.0
    for _ in range(levels - 1):
        edge = edge / (2.0 * N ** (1.0 / D))
        offs = rng.uniform(-0.5, 0.5, size=(len(pts), N, 3)) * edge
        pts = (pts[:, None, :] + offs).reshape(-1, 3)
    return np.mod(pts, 1.0)


def fractal_cloud_grid(n: int = 200, N: int = 32, D: float = 2.3, levels: int = 4, tau: float = 2.0,
                       seed: int = 1556, directions: int = 4096) -> np.ndarray:
    """Density of the fractal cloud on n^3 cells over [-1, 1]^3: proportional to the
    number of points per cell, scaled so that the optical depth from the centre to the
    cube's surface, averaged over directions, is `tau` (the paper's tau_cube).  The
    average is taken over a seeded set of uniform directions, each ray integrated cell
    by cell (exact segment lengths) in float64."""
    pts = fractal_cloud_points(N, D, levels, seed)
    idx = np.minimum((pts * n).astype(np.int64), n - 1)
    counts = np.zeros((n, n, n), dtype=np.float64)
    np.add.at(counts, (idx[:, 2], idx[:, 1], idx[:, 0]), 1.0)
    rng = np.random.Generator(np.random.Philox(seed + 1))
    v = rng.normal(size=(directions, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    taus = np.array([_ray_sum(counts, d) for d in v])
    k = counts * (tau / taus.mean())
    return np.ascontiguousarray(k.astype(np.float32))


def _ray_sum(grid: np.ndarray, d: np.ndarray) -> float:
    """Sum of cell value x segment length along the ray from the centre of [-1, 1]^3
    to its surface (cell faces crossed in order of distance)."""
    n = grid.shape[0]
    h = 2.0 / n
    ts = [0.0]
    for a in range(3):
        if d[a] != 0.0:
            faces = -1.0 + h * np.arange(n + 1)
            t = (faces - 0.0) / d[a]
            ts.extend(t[t > 0].tolist())
    t_exit = min(1.0 / abs(d[a]) for a in range(3) if d[a] != 0.0)
    ts = np.unique(np.clip(np.array(ts), 0.0, t_exit))
    mid = 0.5 * (ts[1:] + ts[:-1])
    seg = ts[1:] - ts[:-1]
    p = mid[:, None] * d[None, :]
    c = np.clip(((p + 1.0) / h).astype(np.int64), 0, n - 1)
    return float(np.sum(grid[c[:, 2], c[:, 1], c[:, 0]] * seg))


# --- workloads ---------------------------------------------------------------------

def homogeneous_sphere_problem(**kw) -> Problem:
    """Point source at the centre of a homogeneous sphere (radius 1, radial tau 0.1,
    albedo 1, isotropic scattering, no polarization), observer at inclination 90
    degrees, 64x64 image."""
    p = Problem(grid=None, sphere_r=1.0, sphere_k=0.1, albedo=1.0, g=0.0, p_l=0.0,
                theta_obs=math.pi / 2, phi_obs=0.0, half_width=1.0, nx=64, ny=64)
    return p.replace(**kw)


_disk_cache: dict = {}


def flared_disk_problem(n: int = 256, generator: str = "sobol", **kw) -> Problem:
    """Point source in a flared disk (rho ~ r^-2 exp(-z^2/2h^2), h = 0.1 r^1.25,
    0.1 <= r <= 1, midplane tau 1), HG g = 0.5, albedo 0.6, p_l = 0.5, observer at
    45 degrees, 256x256 I/Q/U image, on an n^3 grid over [-1, 1]^3."""
    if n not in _disk_cache:
        _disk_cache[n] = flared_disk_grid(n)
    p = Problem(grid=_disk_cache[n], albedo=0.6, g=0.5, p_l=0.5, theta_obs=math.pi / 4, phi_obs=0.0,
                half_width=1.0, nx=256, ny=256, generator=generator)
    return p.replace(**kw)


_clump_cache: dict = {}


def clumpy_problem(n: int = 128, max_orders: int = 20, **kw) -> Problem:
    """Multiple scattering from a point source in an n^3 clumpy envelope (total
    radial tau 5), HG g = 0.6, albedo 0.7, every order forced, roulette below 1e-4,
    four coordinates per order, 512x512 I/Q/U image, observer at 45 degrees."""
    if n not in _clump_cache:
        _clump_cache[n] = clumpy_envelope_grid(n)
    p = Problem(grid=_clump_cache[n], albedo=0.7, g=0.6, p_l=0.5, theta_obs=math.pi / 4, phi_obs=0.0,
                half_width=1.0, nx=512, ny=512, max_orders=max_orders, rr_threshold=1e-4,
                rr_survival=0.1, force="all")
    return p.replace(**kw)


@dataclass
class Instance:
    """One member of a batched run: an observer inclination, a wavelength (albedo, g,
    opacity multiplier) and a packet budget."""

    theta_obs: float
    albedo: float
    g: float
    kscale: float
    n_packets: int
    first_index: int = 1


def batched_instances(n_incl: int = 32, n_wave: int = 8, seed: int = 4, min_log2: int = 18,
                      max_log2: int = 24) -> list[Instance]:
    """n_incl inclinations in [0, 90] degrees x n_wave wavelengths (albedo 0.4-0.9,
    g 0.2-0.7, opacity x0.5-x4 log-spaced), budgets 2^floor(U(min_log2, max_log2))
    drawn from a seeded Philox stream."""
    rng = np.random.Generator(np.random.Philox(seed))
    exps = np.floor(rng.uniform(min_log2, max_log2, size=n_incl * n_wave)).astype(int)
    out = []
    for j in range(n_incl):
        th = math.radians(90.0 * j / max(1, n_incl - 1))
        for l in range(n_wave):
            t = l / max(1, n_wave - 1)
            n = int(2 ** exps[j * n_wave + l])
            # points n .. 2n-1: an aligned block of the sequence (a digitally shifted net)
            out.append(Instance(theta_obs=th, albedo=0.4 + 0.5 * t, g=0.2 + 0.5 * t,
                                kscale=0.5 * 8.0 ** t, n_packets=n, first_index=n))
    return out


_shell_cache: dict = {}


def shell_envelope_problem(n: int = 256, **kw) -> Problem:
    """Point source inside the dust shell (radial tau 0.1), HG g = 0.5, albedo 0.6,
    p_l = 0.5, observer at the pole, 256x256 image."""
    if n not in _shell_cache:
        _shell_cache[n] = shell_envelope_grid(n)
    p = Problem(grid=_shell_cache[n], albedo=0.6, g=0.5, p_l=0.5, theta_obs=0.0, phi_obs=0.0, half_width=1.0,
                nx=256, ny=256)
    return p.replace(**kw)


_fractal_cache: dict = {}


def fractal_cloud_problem(n: int = 200, **kw) -> Problem:
    """Point source at the centre of the fractal cloud (n^3 cells, N = 32 points per
    level, four levels, fractal dimension 2.3, average radial tau 2), single
    scattering, isotropic unpolarized dust (albedo 1, g = 0), observer at 60 degrees,
    200x200 image."""
    if n not in _fractal_cache:
        _fractal_cache[n] = fractal_cloud_grid(n)
    p = Problem(grid=_fractal_cache[n], albedo=1.0, g=0.0, p_l=0.0, theta_obs=math.radians(60.0), phi_obs=0.0,
                half_width=1.0, nx=200, ny=200)
    return p.replace(**kw)


def finite_star_disk_problem(n: int = 256, **kw) -> Problem:
    """The flared disk lit by a finite star (R* = 0.05, linear limb darkening
    u = 0.6, inverse number order)."""
    p = flared_disk_problem(n=n, source="sphere", star_r=0.05, limb_u=0.6, emit_order="inverse")
    return p.replace(**kw)
