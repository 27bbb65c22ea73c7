"""The allocation-free single-scattering entry point, for callers that cannot allocate
device memory (a host application that owns all device memory through its own pool,
or code that must not allocate once running).  It must give the same image as the
regular entry points, on consecutive calls that reuse its built-in scratch.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2406_15632_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def _regular(Q, sc, prob, first, count, fb, precision):
    buf = sc.accum_buffer("i64")
    sc.trace(first, count, buf, frac_bits=fb, precision=precision)
    return sc.reduce(buf, 1.0 / count, frac_bits=fb)[0]


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_noalloc_matches_regular_entry_points_on_consecutive_calls(Q, precision):
    import torch

    prob = S.flared_disk_problem(n=32, nx=96, ny=80)
    sc = Q.Scene(prob)
    fb = 40
    out = torch.full((3, prob.ny, prob.nx), float("nan"), dtype=torch.float64, device="cuda")
    for first, count in ((1, 1 << 14), (1 + (1 << 14), 5000)):
        pts = Q.points_desc(prob.generator, prob.dims, first, count)
        Q.qmcrt_trace_single_noalloc(sc.medium, sc.source, sc.dust, sc.obs, pts, sc.opts(precision), fb,
                                     1.0 / count, out.data_ptr(), Q._stream(None))
        ref = _regular(Q, sc, prob, first, count, fb, precision)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_noalloc_rejects_images_beyond_its_scratch(Q):
    import torch

    prob = S.flared_disk_problem(n=16, nx=1024, ny=1024)
    sc = Q.Scene(prob)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(Q.QmcrtError) as e:
        Q.qmcrt_trace_single_noalloc(sc.medium, sc.source, sc.dust, sc.obs, Q.points_desc("sobol", 3, 1, 64),
                                     sc.opts(), 40, 1.0, out.data_ptr(), 0)
    assert e.value.code == Q.ERR_INVALID_ARG and "pixels" in str(e.value)


def _cudart():
    import ctypes

    for name in ("/usr/local/cuda/lib64/libcudart.so", "libcudart.so", "libcudart.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("no CUDA runtime library to capture a stream with")


def _captured_nodes(rt, stream, call):
    """Number of graph nodes a call enqueues on `stream`, by capturing it (relaxed mode)."""
    import ctypes

    h = ctypes.c_void_p(stream)
    assert rt.cudaStreamBeginCapture(h, 2) == 0  # cudaStreamCaptureModeRelaxed
    try:
        call()
    finally:
        graph = ctypes.c_void_p()
        assert rt.cudaStreamEndCapture(h, ctypes.byref(graph)) == 0
    n = ctypes.c_size_t(0)
    assert rt.cudaGraphGetNodes(graph, None, ctypes.byref(n)) == 0
    assert rt.cudaGraphDestroy(graph) == 0
    return n.value


def test_noalloc_rejects_bad_arguments_before_enqueuing(Q):
    """A rejected call enqueues nothing (the scratch clear comes after every check):
    captured on a stream it adds no graph node, while an accepted call adds its clear,
    trace and reduction."""
    import torch

    prob = S.flared_disk_problem(n=16, nx=32, ny=32)
    sc = Q.Scene(prob)
    out = torch.zeros((3, 32, 32), dtype=torch.float64, device="cuda")
    pts = Q.points_desc("sobol", 3, 1, 256)
    Q.qmcrt_trace_single_noalloc(sc.medium, sc.source, sc.dust, sc.obs, pts, sc.opts(), 40, 1.0 / 256,
                                 out.data_ptr(), 0)  # the first call, outside any capture
    torch.cuda.synchronize()
    rt = _cudart()
    s = torch.cuda.Stream()
    bad_dust = Q.qmcrt_dust.from_buffer_copy(sc.dust)
    bad_dust.g = 1.5
    bad_pts = Q.points_desc("sobol", 2, 1, 256)  # the point source needs 3 coordinates
    for args in ((sc.medium, sc.source, bad_dust, sc.obs, pts, sc.opts(), 40),
                 (sc.medium, sc.source, sc.dust, sc.obs, pts, sc.opts(), 63),
                 (sc.medium, sc.source, sc.dust, sc.obs, bad_pts, sc.opts(), 40)):
        def bad():
            with pytest.raises(Q.QmcrtError) as e:
                Q.qmcrt_trace_single_noalloc(*args, 1.0, out.data_ptr(), s.cuda_stream)
            assert e.value.code == Q.ERR_INVALID_ARG
        assert _captured_nodes(rt, s.cuda_stream, bad) == 0

    def good():
        Q.qmcrt_trace_single_noalloc(sc.medium, sc.source, sc.dust, sc.obs, pts, sc.opts(), 40, 1.0 / 256,
                                     out.data_ptr(), s.cuda_stream)
    assert _captured_nodes(rt, s.cuda_stream, good) >= 3
    torch.cuda.synchronize()
