"""The C-ABI library builds, loads and exports every entry point the header declares;
host-side argument validation rejects bad calls before any device work (these calls
never reach the GPU, so they run without one)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2406_15632_gb300 import build as B
from paper_2406_15632_gb300 import qmcrt as Q

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qmcrt.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Q.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(qmcrt_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_four_path_calls():
    names = declared_functions()
    for n in ("qmcrt_generate_points", "qmcrt_trace_single", "qmcrt_trace_multiple", "qmcrt_image_reduce"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(Q.EXPORTED) == sorted(declared_functions())
    assert lib.qmcrt_abi_version() == 3


STRUCTS = ["qmcrt_points_desc", "qmcrt_medium", "qmcrt_source", "qmcrt_dust", "qmcrt_observer", "qmcrt_image",
           "qmcrt_trace_opts", "qmcrt_instance", "qmcrt_batch_config", "qmcrt_gemm_epilogue",
           "qmcrt_warp", "qmcrt_adam", "qmcrt_host_io"]


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """Compile the header with the host C compiler and compare every struct's size and
    field offsets with the ctypes mirrors used by the binding."""
    import subprocess

    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qmcrt.h"', "int main(void) {"]
    for sname in STRUCTS:
        cls = getattr(Q, sname)
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname}.{fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for sname in STRUCTS:
        cls = getattr(Q, sname)
        assert int(got[sname]) == C.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert int(got[f"{sname}.{fname}"]) == getattr(cls, fname).offset, (sname, fname)


def _expect(code, fn, *args):
    with pytest.raises(Q.QmcrtError) as e:
        fn(*args)
    assert e.value.code == code, str(e.value)
    return str(e.value)


def test_points_validation(lib):
    d = Q.points_desc("sobol", 3, 1, 16)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_generate_points, d, 0)  # NULL output
    fake = 0x1000  # never dereferenced: validation fails first
    for bad in (Q.points_desc("sobol", 0, 1, 16), Q.points_desc("sobol", 257, 1, 16),
                Q.points_desc("sobol", 3, 0, 16), Q.points_desc("halton", 3, 1, 16, fmt="u32"),
                Q.points_desc("sobol", 3, 2 ** 32 - 4, 16), Q.points_desc("hammersley", 2, 1, 16, total_n=8)):
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_generate_points, bad, fake)
    d = Q.points_desc("sobol", 3, 1, 16)
    d.struct_size = 40
    assert "ABI" in _expect(Q.ERR_INVALID_ARG, Q.qmcrt_generate_points, d, fake)
    d = Q.points_desc("sobol", 3, 1, 16)
    d.kind = 9
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_generate_points, d, fake)


def _descs(**over):
    medium = Q._new(Q.qmcrt_medium, kind=Q.MEDIUM_SPHERE, kscale=1.0, sphere_r=1.0, sphere_k=0.1)
    source = Q._new(Q.qmcrt_source, kind=Q.SOURCE_POINT)
    dust = Q._new(Q.qmcrt_dust, albedo=1.0, g=0.0, p_l=0.0)
    obs = Q._new(Q.qmcrt_observer, splat=0, theta=1.0, phi=0.0, half_width=1.0, nx=8, ny=8)
    pts = Q.points_desc("sobol", 3, 1, 64)
    opts = Q._new(Q.qmcrt_trace_opts, precision=0, tau_min=1e-12, max_orders=1, rr_survival=0.1)
    img = Q._new(Q.qmcrt_image, accum=0, d_accum=0x1000, n_images=1, frac_bits=40)
    d = dict(medium=medium, source=source, dust=dust, obs=obs, pts=pts, opts=opts, img=img)
    for k, v in over.items():
        obj, field = k.split("__")
        setattr(d[obj], field, v)
    return d


BAD_TRACE = [
    dict(dust__g=1.0), dict(dust__albedo=1.5), dict(dust__p_l=-0.1), dict(obs__nx=0), dict(obs__half_width=0.0),
    dict(obs__splat=3), dict(pts__first_index=0), dict(pts__dims=2), dict(img__d_accum=None), dict(img__frac_bits=63),
    dict(img__accum=5), dict(img__n_images=2), dict(opts__precision=7), dict(opts__block_size=48),
    dict(medium__kind=0), dict(medium__kscale=0.0), dict(source__kind=1), dict(opts__tau_min=-1.0),
    dict(obs__d_tail=0x7000),  # a tail map over an analytic sphere
]


@pytest.mark.parametrize("over", BAD_TRACE)
def test_trace_single_validation(lib, over):
    d = _descs(**over)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_single, d["medium"], d["source"], d["dust"], d["obs"], d["pts"],
            d["opts"], d["img"], 0, 0)


@pytest.mark.parametrize("over", BAD_TRACE[:6])
def test_trace_observers_validation(lib, over):
    """The observer-set entry point rejects what the single-observer one rejects, an
    observer count outside 1..16, and observers of different image shape."""
    d = _descs(**over)

    def call(obs_list, n):
        arr = (Q.qmcrt_observer * max(len(obs_list), 1))(*obs_list)
        Q.qmcrt_trace_observers(d["medium"], d["source"], d["dust"], arr, n, d["pts"], d["opts"], d["img"], 0)

    with pytest.raises(Q.QmcrtError) as e:
        call([d["obs"], _descs()["obs"]], 2)
    assert e.value.code == Q.ERR_INVALID_ARG
    good = _descs()
    for obs_list, n in (([good["obs"]], 0), ([good["obs"]] * 17, 17)):
        with pytest.raises(Q.QmcrtError) as e:
            Q.qmcrt_trace_observers(good["medium"], good["source"], good["dust"],
                                    (Q.qmcrt_observer * len(obs_list))(*obs_list), n, good["pts"], good["opts"],
                                    good["img"], 0)
        assert e.value.code == Q.ERR_INVALID_ARG
    wide = _descs(obs__nx=16)["obs"]
    with pytest.raises(Q.QmcrtError) as e:
        Q.qmcrt_trace_observers(good["medium"], good["source"], good["dust"],
                                (Q.qmcrt_observer * 2)(good["obs"], wide), 2, good["pts"], good["opts"], good["img"], 0)
    assert e.value.code == Q.ERR_INVALID_ARG


def test_trace_multiple_validation(lib):
    d = _descs(opts__max_orders=3)
    d["pts"].dims = 11  # needs 12
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_multiple, d["medium"], d["source"], d["dust"], d["obs"], d["pts"],
            d["opts"], d["img"], 0)
    d = _descs(opts__max_orders=3, opts__rr_survival=0.0)
    d["pts"].dims = 12
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_multiple, d["medium"], d["source"], d["dust"], d["obs"], d["pts"],
            d["opts"], d["img"], 0)
    # a finite star needs its two extra emission coordinates after all orders' ones
    d = _descs(opts__max_orders=3, source__kind=1, source__radius=0.1)
    d["pts"].dims = 13
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_multiple, d["medium"], d["source"], d["dust"], d["obs"], d["pts"],
            d["opts"], d["img"], 0)


def test_image_reduce_validation(lib):
    img = Q._new(Q.qmcrt_image, accum=0, d_accum=0x1000, n_images=1, frac_bits=40)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_image_reduce, img, 8, 8, 1, 1.0, 0)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_image_reduce, img, 0, 8, 1, 1.0, 0x2000)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_image_reduce, img, 8, 8, 0, 1.0, 0x2000)


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(Q.QmcrtError):
        Q._lib_saved = Q._lib
        Q._lib = None
        try:
            Q.load(str(tmp_path / "nope.so"))
        finally:
            Q._lib = Q._lib_saved


def test_sobol_byte_table_gives_the_oracle_points():
    """The byte-grouped direction numbers the kernels use for the leading dimensions: the
    XOR of one entry per byte of gray(i) is the Sobol coordinate the oracle computes."""
    from oracle import oracle as O

    T = B.sobol_byte_table(B.sobol_direction_table(B.SOBOL_BYTE_DIMS))
    idx = np.concatenate([np.arange(4096), np.random.default_rng(3).integers(0, 1 << 32, 4096)]).astype(np.uint64)
    g = idx ^ (idx >> np.uint64(1))
    got = np.zeros((idx.size, B.SOBOL_BYTE_DIMS), dtype=np.uint64)
    for d in range(B.SOBOL_BYTE_DIMS):
        for b in range(4):
            got[:, d] ^= np.asarray(T[d][b], dtype=np.uint64)[(g >> np.uint64(8 * b)) & np.uint64(255)]
    for lo in (0, 4096):
        ref = O.generate_points("sobol", B.SOBOL_BYTE_DIMS, 0, 4096, "u32") if lo == 0 else np.stack(
            [O.generate_points("sobol", B.SOBOL_BYTE_DIMS, int(i), 1, "u32")[0] for i in idx[4096:4160]])
        n = ref.shape[0]
        assert np.array_equal(got[lo:lo + n], ref.astype(np.uint64))


def test_default_frac_bits_never_overflows_and_is_the_largest_such_scale(lib):
    """The library's scale F: n x (contributions per pixel and packet) x bound x 2^F stays
    below 2^62, and F + 1 would not (F is the largest safe scale); F never grows with n."""
    from paper_2406_15632_gb300 import scenes as S

    cases = ((S.flared_disk_problem(n=8), 1 << 28, 1.0), (S.homogeneous_sphere_problem(), 1 << 16, 1.0),
             (S.clumpy_problem(n=8), 1 << 24, 1.0), (S.clumpy_problem(n=8, per_order=True), 1 << 24, 1.0),
             (S.clumpy_problem(n=8), 1 << 22, 1000.0),
             (S.finite_star_disk_problem(n=8), 1 << 23, 1.0))
    for prob, n, wb in cases:
        fb = Q.default_frac_bits(prob, n, wb)
        per = prob.max_orders if prob.max_orders > 1 and not prob.per_order else 1
        total = n * per * Q.contribution_bound(prob) * wb
        assert 0 <= fb <= 62
        assert total * 2.0 ** fb <= 2.0 ** 62
        assert fb == 62 or total * 2.0 ** (fb + 1) > 2.0 ** 62
        assert Q.default_frac_bits(prob, 4 * n, wb) <= fb


def test_contribution_bound_and_frac_bits_validation(lib):
    d = _descs()
    out = C.c_double()
    assert Q.qmcrt_contribution_bound(d["source"], d["dust"], d["opts"], False) > 0
    for over in (dict(dust__g=1.0), dict(dust__albedo=-0.5), dict(dust__p_l=2.0)):
        b = _descs(**over)
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_contribution_bound, b["source"], b["dust"], b["opts"], False)
    b = _descs(opts__max_orders=0)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_contribution_bound, b["source"], b["dust"], b["opts"], True)
    b = _descs()
    b["dust"].struct_size = 8
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_contribution_bound, b["source"], b["dust"], b["opts"], False)
    assert lib.qmcrt_contribution_bound(C.byref(d["source"]), C.byref(d["dust"]), C.byref(d["opts"]), 0,
                                        None) == Q.ERR_INVALID_ARG
    for wb in (0.5, float("inf"), float("nan")):
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_default_frac_bits, d["source"], d["dust"], d["opts"], False, 1 << 20, wb)
    del out


def test_render_single_host_validation(lib):
    """The host-buffer render rejects bad buffers before anything is enqueued (these
    calls never reach the GPU)."""
    d = _descs()
    io = Q._new(Q.qmcrt_host_io, h_k=None, d_k=None, d_accum=0x1000, d_image=0x2000, h_image=0x3000)

    def call(dd, io_):
        Q.qmcrt_render_single_host(dd["medium"], dd["source"], dd["dust"], dd["obs"], dd["pts"], dd["opts"], io_,
                                   40, 1.0, 0)
    for field in ("d_accum", "d_image", "h_image"):
        bad = Q.qmcrt_host_io.from_buffer_copy(io)
        setattr(bad, field, None)
        _expect(Q.ERR_INVALID_ARG, call, d, bad)
    bad = Q.qmcrt_host_io.from_buffer_copy(io)
    bad.struct_size = 16
    _expect(Q.ERR_INVALID_ARG, call, d, bad)
    bad = Q.qmcrt_host_io.from_buffer_copy(io)
    bad.h_k = 0x4000  # a grid for a sphere medium
    _expect(Q.ERR_INVALID_ARG, call, d, bad)
    g = _descs(medium__kind=0, medium__d_k=0x5000, medium__nx=4, medium__ny=4, medium__nz=4, medium__pad=8)
    for a in range(3):
        g["medium"].lo[a], g["medium"].hi[a] = -1.0, 1.0
    bad = Q.qmcrt_host_io.from_buffer_copy(io)
    bad.h_k = 0x4000  # a padded grid needs d_k
    _expect(Q.ERR_INVALID_ARG, call, g, bad)
    bad.d_k = 0x5000  # ... distinct from the padded grid
    _expect(Q.ERR_INVALID_ARG, call, g, bad)
    # a bound map is rebuilt from the new grid: its workspace is checked before anything runs
    g2 = _descs(medium__kind=0, medium__d_k=0x5000, medium__nx=4, medium__ny=4, medium__nz=4, medium__pad=8,
                medium__d_sky=0x6000, medium__sky_m=16)
    for a in range(3):
        g2["medium"].lo[a], g2["medium"].hi[a] = -1.0, 1.0
    ok = Q.qmcrt_host_io.from_buffer_copy(io)
    ok.h_k, ok.d_k = 0x4000, 0x7000
    for ws, nbytes in ((None, 0), (0x8000, 16), (0x8010, 1 << 20)):
        b = Q.qmcrt_host_io.from_buffer_copy(ok)
        b.d_sky_ws, b.sky_ws_bytes = ws, nbytes
        _expect(Q.ERR_INVALID_ARG, call, g2, b)
    # so is a tail map of the observer's direction
    g3 = _descs(medium__kind=0, medium__d_k=0x5000, medium__nx=4, medium__ny=4, medium__nz=4, medium__pad=8,
                obs__d_tail=0x9000)
    for a in range(3):
        g3["medium"].lo[a], g3["medium"].hi[a] = -1.0, 1.0
    for ws, nbytes in ((None, 0), (0x8000, 16), (0x8010, 1 << 20)):
        b = Q.qmcrt_host_io.from_buffer_copy(ok)
        b.d_tail_ws, b.tail_ws_bytes = ws, nbytes
        _expect(Q.ERR_INVALID_ARG, call, g3, b)
    for over in BAD_TRACE[:8]:
        _expect(Q.ERR_INVALID_ARG, call, _descs(**over), io)


@pytest.mark.parametrize("g,albedo,p_l", [(0.6, 0.7, 0.5), (-0.4, 1.0, 1.0), (0.0, 0.9, 0.3)])
def test_contribution_bound_holds_through_scattering_and_peel_off(g, albedo, p_l):
    """Random packets pushed through the oracle's scattering and peel-off steps: no
    contribution of order k exceeds the bound of a problem with k orders, and the
    bound is reached within a factor of a few at the first order (it is tight where
    the fixed-point scale needs it)."""
    from oracle import oracle as O
    from paper_2406_15632_gb300 import scenes as S

    rng = np.random.default_rng(3)
    K = 6
    prob = S.homogeneous_sphere_problem(sphere_k=1e-9, g=g, albedo=albedo, p_l=p_l, max_orders=K)
    worst = np.zeros(K + 1)
    for _ in range(300):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a = np.cross(n, [0.0, 0.0, 1.0]) if abs(n[2]) < 0.9 else np.cross(n, [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        S3 = np.array([1.0, 0.0, 0.0])
        for k in range(1, K + 1):
            if k > 1:
                n, a, S3 = O.scatter_packet(prob, rng.uniform(), rng.uniform(), n, a, S3)
            S3 = S3 * albedo  # forcing weight <= 1 taken as 1
            ok, out = O.peel_packet(prob, [0.0, 0.0, 0.0], n, a, S3)
            if ok:
                worst[k] = max(worst[k], np.abs(out[:3]).max())
    for k in range(1, K + 1):
        assert worst[k] <= Q.contribution_bound(prob.replace(max_orders=k)) * (1 + 1e-12), k
    assert worst[1] >= 0.05 * Q.contribution_bound(prob.replace(max_orders=1))


def test_sky_bound_validation(lib):
    lo, hi = [-1.0] * 3, [1.0] * 3
    ws = Q.qmcrt_sky_workspace_bytes(4, 4, 4, lo, hi, 0.0)
    assert ws == 2 * ((6 ** 3 * 4 + 255) // 256 * 256)  # two grids grown by one layer
    assert Q.qmcrt_sky_workspace_bytes(4, 4, 4, lo, hi, 0.6) > ws  # a star grows them further
    assert Q.qmcrt_sky_workspace_bytes(0, 4, 4, lo, hi, 0.0) == 0
    good = [0x1000, 4, 4, 4, lo, hi, 0.0, 16, 0x2000, 0x4000, ws]
    for i, bad in ((0, 0), (8, 0), (9, 0), (9, 0x4010), (10, ws - 1), (1, 0), (5, [1.0, -1.0, 1.0]), (6, -0.1),
                   (6, float("nan")), (7, 0), (7, 4097)):
        a = list(good)
        a[i] = bad
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_sky_bound, *a)
    # a trace rejects a bound map of impossible size
    g = _descs(medium__kind=0, medium__d_k=0x5000, medium__nx=4, medium__ny=4, medium__nz=4, medium__d_sky=0x6000,
               medium__sky_m=0)
    for a in range(3):
        g["medium"].lo[a], g["medium"].hi[a] = -1.0, 1.0
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_single, g["medium"], g["source"], g["dust"], g["obs"], g["pts"],
            g["opts"], g["img"], 0, 0)


def _padded_grid_descs(**over):
    base = dict(medium__kind=Q.MEDIUM_GRID, medium__d_k=0x5000, medium__nx=6, medium__ny=5, medium__nz=7,
                medium__pad=Q.MIN_PAD)
    base.update(over)
    g = _descs(**base)
    for a in range(3):
        g["medium"].lo[a], g["medium"].hi[a] = -1.0, 1.0
    return g


def test_tail_map_validation(lib):
    assert Q.qmcrt_tail_map_bytes(6, 5, 7, 4) == 14 * 13 * 15
    assert Q.qmcrt_tail_map_bytes(0, 5, 7, 4) == 0
    ws = Q.qmcrt_tail_workspace_bytes(6, 5, 7)
    assert ws == 2 * ((2 * 2 * 2 * 4 + 255) // 256 * 256)  # two arrays of 4^3-cell block values
    assert Q.qmcrt_tail_workspace_bytes(6, 5, 0) == 0
    g = _padded_grid_descs()
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_tail_map, g["medium"], g["obs"], 0, 0x2000, ws)  # no map
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_tail_map, g["medium"], g["obs"], 0x1000, 0, ws)  # no workspace
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_tail_map, g["medium"], g["obs"], 0x1000, 0x2010, ws)  # misaligned
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_tail_map, g["medium"], g["obs"], 0x1000, 0x2000, ws - 1)
    for over in (dict(medium__pad=0), dict(medium__pad=Q.MIN_PAD - 1), dict(medium__kind=Q.MEDIUM_SPHERE),
                 dict(medium__d_k=None), dict(medium__nz=0), dict(obs__theta=float("nan")),
                 dict(obs__phi=float("inf")), dict(medium__struct_size=8), dict(obs__struct_size=8)):
        b = _padded_grid_descs(**over)
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_tail_map, b["medium"], b["obs"], 0x1000, 0x2000, ws)
    b = _padded_grid_descs()
    b["medium"].hi[1] = -1.0
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_tail_map, b["medium"], b["obs"], 0x1000, 0x2000, ws)
    # a trace rejects a tail map on an unpadded grid and a tolerance that is negative or NaN
    for over in (dict(medium__pad=0, obs__d_tail=0x7000), dict(obs__d_tail=0x7000, opts__tail_eps=-1e-9),
                 dict(obs__d_tail=0x7000, opts__tail_eps=float("nan"))):
        b = _padded_grid_descs(**over)
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_single, b["medium"], b["source"], b["dust"], b["obs"], b["pts"],
                b["opts"], b["img"], 0, 0)


def test_batch_validation(lib):
    d = _descs()
    pts = Q.points_desc("sobol", 5, 1, 1)
    cfg = Q._new(Q.qmcrt_batch_config, chunk_log2=16, block_size=256, ctas_per_sm=0, packets_per_thread=4)
    img = Q._new(Q.qmcrt_image, accum=0, d_accum=0x1000, n_images=1, frac_bits=40)
    ws = Q.qmcrt_batch_workspace_bytes(8)
    assert ws >= 8 * 10 and ws % 256 == 0
    args = [d["medium"], d["source"], d["obs"], pts, d["opts"], 0x3000, 8, cfg, 0x4000, ws, img, 0]
    for i, bad in ((5, 0), (6, 0), (8, 0), (9, ws - 8)):
        a = list(args)
        a[i] = bad
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_batch, *a)
    for field, v in (("chunk_log2", 3), ("block_size", 96), ("packets_per_thread", 0), ("ctas_per_sm", -1)):
        c = Q._new(Q.qmcrt_batch_config, chunk_log2=16, block_size=256, ctas_per_sm=0, packets_per_thread=4)
        setattr(c, field, v)
        a = list(args)
        a[7] = c
        _expect(Q.ERR_INVALID_ARG, Q.qmcrt_trace_batch, *a)
    img2 = Q._new(Q.qmcrt_image, accum=1, d_accum=0x1000, n_images=1, frac_bits=40)
    _expect(Q.ERR_INVALID_ARG, Q.qmcrt_batch_reduce, img2, 0x3000, 8, 8, 8, 0x5000)


def test_warp_constants_match_the_oracle_layout():
    from oracle import flow as F

    assert Q.WARP_PARAMS == F.N_PARAMS
    assert Q.WARP_BF16_WEIGHTS == sum(F.LAYOUT[f"W{m}{l}"][1][0] * F.LAYOUT[f"W{m}{l}"][1][1]
                                      for m in range(2) for l in range(4))
    assert Q.Warp.initial(0).numel() == F.N_PARAMS
