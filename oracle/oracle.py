"""Python front of the FP64 CPU oracle (qmcrt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It compiles the C file with
gcc into oracle/_build/ and calls it through ctypes.  It shares no code with the
CUDA path; the only common input is the problem description from the scene module
and the Joe-Kuo direction-number data file that ships with SciPy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmcrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

KINDS = {"sobol": 0, "sobol_owen": 1, "halton": 2, "hammersley": 3, "philox": 4, "niederreiter": 5, "faure": 6}
FORMATS = {"u32": 0, "f32": 1, "f64": 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, IEEE double, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Medium(C.Structure):
    _fields_ = [("kind", C.c_int), ("k", C.POINTER(C.c_float)), ("n", C.c_int * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("kscale", C.c_double),
                ("sphere_r", C.c_double), ("sphere_k", C.c_double)]


class _Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("r", C.c_double), ("limb_u", C.c_double), ("order", C.c_int)]


class _Dust(C.Structure):
    _fields_ = [("albedo", C.c_double), ("g", C.c_double), ("p_l", C.c_double)]


class _Observer(C.Structure):
    _fields_ = [("theta", C.c_double), ("phi", C.c_double), ("half_width", C.c_double),
                ("nx", C.c_int), ("ny", C.c_int), ("splat", C.c_int)]


class _Points(C.Structure):
    _fields_ = [("kind", C.c_int), ("dims", C.c_int), ("seed", C.c_uint64), ("total_n", C.c_uint64),
                ("V", C.POINTER(C.c_uint32))]


class _Problem(C.Structure):
    _fields_ = [("medium", _Medium), ("source", _Source), ("dust", _Dust), ("obs", _Observer),
                ("points", _Points), ("tau_min", C.c_double), ("max_orders", C.c_int),
                ("rr_threshold", C.c_double), ("rr_survival", C.c_double), ("force_all", C.c_int),
                ("per_order", C.c_int)]


_D3 = C.c_double * 3


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u64, i32, dp = C.c_uint64, C.c_int, C.POINTER(C.c_double)
            L.or_sobol_directions.argtypes = [i32, C.POINTER(C.c_int64), C.POINTER(C.c_int64), i32,
                                              C.POINTER(C.c_uint32)]
            L.or_sobol_u32.restype = C.c_uint32
            L.or_sobol_u32.argtypes = [C.POINTER(C.c_uint32), i32, u64]
            L.or_owen_scramble.restype = C.c_uint32
            L.or_owen_scramble.argtypes = [C.c_uint32, C.c_uint32]
            L.or_owen_seed.restype = C.c_uint32
            L.or_owen_seed.argtypes = [u64, i32]
            L.or_radical_inverse.restype = C.c_double
            L.or_radical_inverse.argtypes = [u64, C.c_uint32]
            L.or_prime.restype = C.c_uint32
            L.or_prime.argtypes = [i32]
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.or_generate_points.argtypes = [i32, i32, u64, u64, C.POINTER(C.c_uint32), u64, u64, i32, C.c_void_p]
            L.or_niederreiter_columns.argtypes = [i32, C.POINTER(C.c_uint32)]
            L.or_niederreiter_u32.restype = C.c_uint32
            L.or_niederreiter_u32.argtypes = [C.POINTER(C.c_uint32), i32, u64]
            L.or_faure_base.restype = C.c_uint32
            L.or_faure_base.argtypes = [i32]
            L.or_faure.restype = C.c_double
            L.or_faure.argtypes = [u64, i32, C.c_uint32]
            L.or_hg_cos.restype = C.c_double
            L.or_hg_cos.argtypes = [C.c_double, C.c_double]
            P = C.POINTER(_Problem)
            L.or_trace_single.argtypes = [P, u64, u64, dp, dp, i32]
            L.or_trace_multiple.argtypes = [P, u64, u64, dp, i32]
            L.or_trace_multiple_warped.argtypes = [P, u64, u64, dp, dp, dp, dp, i32]
            L.or_trace_multiple_cells.argtypes = [P, u64, u64, dp, dp]
            L.or_direct_light.argtypes = [P, i32, C.c_double, dp]
            L.or_tau_ray.restype = C.c_double
            L.or_tau_ray.argtypes = [P, dp, dp]
            L.or_ray_cells.argtypes = [P, dp, dp, C.c_double, dp]
            L.or_march_ray.argtypes = [P, dp, dp, C.c_double, dp]
            L.or_scatter_packet.argtypes = [P, C.c_double, C.c_double, dp, dp, dp]
            L.or_peel_packet.argtypes = [P, dp, dp, dp, dp, dp]
            L.or_emit_packet.restype = C.c_double
            L.or_emit_packet.argtypes = [P, u64, dp, dp, dp, dp]
            _lib = L
    return _lib


# --- Sobol direction numbers ----------------------------------------------------------

_V_cache: dict = {}


def joe_kuo_data():
    """Joe & Kuo (2008) primitive polynomials and initial direction values, read from
    the data file that ships with SciPy (poly with leading and trailing ones; vinit
    holds m_1.. m_s)."""
    import scipy
    d = np.load(os.path.join(os.path.dirname(scipy.__file__), "stats", "_sobol_direction_numbers.npz"))
    return np.ascontiguousarray(d["poly"], dtype=np.int64), np.ascontiguousarray(d["vinit"], dtype=np.int64)


def sobol_directions(dims: int) -> np.ndarray:
    if dims not in _V_cache:
        poly, vinit = joe_kuo_data()
        V = np.zeros((dims, 32), dtype=np.uint32)
        rc = lib().or_sobol_directions(dims, poly.ctypes.data_as(C.POINTER(C.c_int64)),
                                       vinit.ctypes.data_as(C.POINTER(C.c_int64)), vinit.shape[1],
                                       V.ctypes.data_as(C.POINTER(C.c_uint32)))
        if rc != 0:
            raise RuntimeError(f"direction numbers: rc={rc}")
        _V_cache[dims] = V
    return _V_cache[dims]


_N_cache: dict = {}


def niederreiter_columns(dims: int) -> np.ndarray:
    """[dims][32] generator-matrix columns of the base-2 Niederreiter sequence."""
    if dims not in _N_cache:
        V = np.zeros((dims, 32), dtype=np.uint32)
        rc = lib().or_niederreiter_columns(dims, V.ctypes.data_as(C.POINTER(C.c_uint32)))
        if rc != 0:
            raise RuntimeError(f"niederreiter columns: rc={rc}")
        _N_cache[dims] = V
    return _N_cache[dims]


def digital_table(kind: str, dims: int) -> np.ndarray:
    """The 32-bit column table a generator of this kind reads (Sobol or Niederreiter)."""
    return niederreiter_columns(max(dims, 1)) if kind == "niederreiter" else sobol_directions(max(dims, 1))


def faure_base(dims: int) -> int:
    return lib().or_faure_base(dims)


def faure(i: int, d: int, b: int) -> float:
    return lib().or_faure(i, d, b)


# --- points -------------------------------------------------------------------------------

def generate_points(kind: str, dims: int, first: int, count: int, fmt: str = "f64", seed: int = 0,
                    total_n: int = 0) -> np.ndarray:
    """Row-major [count][dims] points with indices first .. first+count-1."""
    dt = {"u32": np.uint32, "f32": np.float32, "f64": np.float64}[fmt]
    out = np.zeros((count, dims), dtype=dt)
    V = digital_table(kind, dims)
    rc = lib().or_generate_points(KINDS[kind], dims, seed, total_n, V.ctypes.data_as(C.POINTER(C.c_uint32)),
                                  first, count, FORMATS[fmt], out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle generate_points rc={rc}")
    return out


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def radical_inverse(i: int, b: int) -> float:
    return lib().or_radical_inverse(i, b)


def owen_scramble(x: int, seed_d: int) -> int:
    return lib().or_owen_scramble(x, seed_d)


def owen_seed(seed: int, d: int) -> int:
    return lib().or_owen_seed(seed, d)


def prime(n: int) -> int:
    return lib().or_prime(n)


def hg_cos(g: float, v: float) -> float:
    return lib().or_hg_cos(g, v)


# --- problems -----------------------------------------------------------------------------

class _Holder:
    """Keeps the arrays a _Problem points to alive."""

    def __init__(self, prob):
        self.prob = prob
        s = _Problem()
        m = s.medium
        if prob.grid is not None:
            self.grid = np.ascontiguousarray(prob.grid, dtype=np.float32)
            m.kind = 0
            m.k = self.grid.ctypes.data_as(C.POINTER(C.c_float))
            nz, ny, nx = self.grid.shape
            m.n[0], m.n[1], m.n[2] = nx, ny, nz
        else:
            self.grid = None
            m.kind = 1
        for a in range(3):
            m.lo[a] = prob.lo[a]
            m.hi[a] = prob.hi[a]
        m.kscale = prob.kscale
        m.sphere_r = prob.sphere_r
        m.sphere_k = prob.sphere_k
        s.source.kind = 0 if prob.source == "point" else 1
        s.source.r = prob.star_r
        s.source.limb_u = prob.limb_u
        s.source.order = 0 if prob.emit_order == "direct" else 1
        s.dust.albedo, s.dust.g, s.dust.p_l = prob.albedo, prob.g, prob.p_l
        s.obs.theta, s.obs.phi, s.obs.half_width = prob.theta_obs, prob.phi_obs, prob.half_width
        s.obs.nx, s.obs.ny = prob.nx, prob.ny
        s.obs.splat = 0 if prob.splat == "nearest" else 1
        self.V = digital_table(prob.generator, prob.dims)
        s.points.kind = KINDS[prob.generator]
        s.points.dims = prob.dims
        s.points.seed = prob.seed
        s.points.total_n = prob.total_n
        s.points.V = self.V.ctypes.data_as(C.POINTER(C.c_uint32))
        s.tau_min = prob.tau_min
        s.max_orders = prob.max_orders
        s.rr_threshold = prob.rr_threshold
        s.rr_survival = prob.rr_survival
        s.force_all = 1 if prob.force == "all" else 0
        s.per_order = 1 if prob.per_order else 0
        self.s = s

    @property
    def ptr(self):
        return C.byref(self.s)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def trace_single(prob, first: int, count: int, log: bool = False, nthreads: int | None = None):
    """Raw image sums [3][ny][nx] (not divided by N) of packets first..first+count-1,
    and optionally the per-packet log [count][11]: scattering x, y, z, peel-off I, Q, U,
    sky x, y, status, grid cells visited, and of those the cells the march to the scattering
    point visited."""
    h = _Holder(prob)
    img = np.zeros((3, prob.ny, prob.nx), dtype=np.float64)
    lg = np.zeros((count, 11), dtype=np.float64) if log else None
    rc = lib().or_trace_single(h.ptr, first, count, img.ctypes.data_as(C.POINTER(C.c_double)),
                               lg.ctypes.data_as(C.POINTER(C.c_double)) if log else None,
                               nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"oracle trace_single rc={rc}")
    return (img, lg) if log else img


def trace_multiple(prob, first: int, count: int, nthreads: int | None = None):
    """Raw image sums [n_images][3][ny][nx] for multiple scattering."""
    h = _Holder(prob)
    img = np.zeros((prob.n_images, 3, prob.ny, prob.nx), dtype=np.float64)
    rc = lib().or_trace_multiple(h.ptr, first, count, img.ctypes.data_as(C.POINTER(C.c_double)),
                                 nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"oracle trace_multiple rc={rc}")
    return img


def trace_multiple_warped(prob, first: int, count: int, x=None, logj=None, train_log: bool = False,
                          nthreads: int | None = None):
    """Multiple scattering with the first-order coordinates of packet j set to x[j]
    and its weight multiplied by exp(logj[j]).  Returns the raw image sums and, if
    asked, the per-packet log [count][5] (coordinates; sum and L2 norm of the in-image
    peel-off intensities)."""
    h = _Holder(prob)
    img = np.zeros((prob.n_images, 3, prob.ny, prob.nx), dtype=np.float64)
    dp = C.POINTER(C.c_double)
    xa = None if x is None else np.ascontiguousarray(x, dtype=np.float64).reshape(count, 3)
    la = None if logj is None else np.ascontiguousarray(logj, dtype=np.float64).reshape(count)
    tl = np.zeros((count, 5), dtype=np.float64) if train_log else None
    ptr = lambda a: a.ctypes.data_as(dp) if a is not None else None
    rc = lib().or_trace_multiple_warped(h.ptr, first, count, ptr(xa), ptr(la), img.ctypes.data_as(dp), ptr(tl),
                                        nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"oracle trace_multiple_warped rc={rc}")
    return (img, tl) if train_log else img


def direct_light(prob, subsamples: int = 4, weight: float = 1.0):
    """Direct light of the source as an image [3][ny][nx] (Stokes I only), times weight."""
    h = _Holder(prob)
    img = np.zeros((3, prob.ny, prob.nx), dtype=np.float64)
    rc = lib().or_direct_light(h.ptr, subsamples, weight, img.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise RuntimeError(f"oracle direct_light rc={rc}")
    return img


def multiple_cells(prob, first: int, count: int):
    """Grid cells visited per packet by the multiple-scattering tracer (one thread):
    [count][2], all walks and, of those, the marches of forced steps."""
    h = _Holder(prob)
    img = np.zeros((prob.n_images, 3, prob.ny, prob.nx), dtype=np.float64)
    cells = np.zeros((count, 2), dtype=np.float64)
    dp = C.POINTER(C.c_double)
    rc = lib().or_trace_multiple_cells(h.ptr, first, count, img.ctypes.data_as(dp), cells.ctypes.data_as(dp))
    if rc != 0:
        raise RuntimeError(f"oracle multiple_cells rc={rc}")
    return cells


def _vec(v):
    return _D3(*[float(x) for x in v])


def tau_ray(prob, p, d) -> float:
    h = _Holder(prob)
    return lib().or_tau_ray(h.ptr, _vec(p), _vec(d))


def ray_cells(prob, points, d, eps: float):
    """For walks from each of points [n][3] along d: the cells each visits, and how many
    come before the optical depth still ahead is at most eps (what a walk allowed to leave
    out eps must visit); int arrays [n][2]."""
    h = _Holder(prob)
    out = _D3()
    dv = _vec(d)
    res = np.zeros((len(points), 2), dtype=np.int64)
    for j, p in enumerate(points):
        if lib().or_ray_cells(h.ptr, _vec(p), dv, float(eps), out) != 0:
            raise RuntimeError("oracle ray_cells needs a grid medium")
        res[j] = int(out[0]), int(out[1])
    return res


def march_ray(prob, p, d, tau):
    h = _Holder(prob)
    q = _D3()
    hit = lib().or_march_ray(h.ptr, _vec(p), _vec(d), float(tau), q)
    return bool(hit), np.array(list(q))


def scatter_packet(prob, u, v, n, a, S):
    h = _Holder(prob)
    nn, aa, SS = _vec(n), _vec(a), _vec(S)
    lib().or_scatter_packet(h.ptr, float(u), float(v), nn, aa, SS)
    return np.array(list(nn)), np.array(list(aa)), np.array(list(SS))


def peel_packet(prob, pos, n, a, S):
    """(ok, [I, Q, U, sky_x, sky_y]) of the peel-off of one packet."""
    h = _Holder(prob)
    out = (C.c_double * 5)()
    ok = lib().or_peel_packet(h.ptr, _vec(pos), _vec(n), _vec(a), _vec(S), out)
    return bool(ok), np.array(list(out))


def emit_packet(prob, i):
    h = _Holder(prob)
    pos, d, e = _D3(), _D3(), _D3()
    w = C.c_double()
    depth = lib().or_emit_packet(h.ptr, i, pos, d, e, C.byref(w))
    return np.array(list(pos)), np.array(list(d)), np.array(list(e)), w.value, depth
