"""Multiple scattering order by order with live packets regrouped between orders: the
same images as the one-kernel tracer, bit for bit in fixed point, for every forcing
mode, source and point set; the same training log with a learned warp; any chunking
of the packets by the workspace size."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

pytestmark = pytest.mark.gpu

MULTI = S.clumpy_problem(n=24, max_orders=8, nx=40, ny=36, per_order=True, half_width=0.9)
CASES = {
    "force_all": MULTI,
    "force_first": MULTI.replace(force="first", rr_threshold=0.0),
    "roulette_heavy": MULTI.replace(per_order=False, rr_threshold=0.05, rr_survival=0.3),
    "owen": MULTI.replace(per_order=False, generator="sobol_owen", seed=4),
    "halton": MULTI.replace(per_order=False, generator="halton"),
    "star_inverse": MULTI.replace(per_order=False, source="sphere", star_r=0.06, limb_u=0.6),
    "star_direct": MULTI.replace(source="sphere", star_r=0.06, limb_u=0.6, emit_order="direct"),
    "sphere": S.homogeneous_sphere_problem(sphere_k=0.8, max_orders=12, g=0.3, p_l=0.4, per_order=True),
}


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def _both(Q, prob, first, count, precision, ws_packets=None, fb=36):
    import torch

    sc = Q.Scene(prob)
    a = sc.accum_buffer("i64")
    sc.trace(first, count, a, frac_bits=fb, precision=precision)
    b = sc.accum_buffer("i64")
    ws = sc.wavefront_workspace(ws_packets or count, precision)
    sc.trace_wavefront(first, count, b, ws, frac_bits=fb, precision=precision)
    torch.cuda.synchronize()
    return a, b


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("name", list(CASES))
def test_wavefront_equals_one_kernel_tracer(Q, name, precision):
    import torch

    a, b = _both(Q, CASES[name], 1, 1 << 13, precision)
    assert torch.equal(a, b)
    assert bool((a != 0).any())


def test_wavefront_chunks_by_workspace(Q):
    """A workspace for 2^11 packets splits 2^14 + 777 packets at aligned blocks."""
    import torch

    a, b = _both(Q, CASES["force_all"], 3000, (1 << 14) + 777, "f32", ws_packets=1 << 11)
    assert torch.equal(a, b)


def test_wavefront_fp64_matches_oracle(Q):
    import torch

    prob = CASES["star_direct"]
    sc = Q.Scene(prob)
    buf = sc.accum_buffer("f64")
    ws = sc.wavefront_workspace(4096, "f64")
    sc.trace_wavefront(1, 4096, buf, ws, accum="f64", precision="f64")
    torch.cuda.synchronize()
    ref = O.trace_multiple(prob, 1, 4096)
    got = buf[0].cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_wavefront_learned_warp_and_training_log(Q):
    import torch

    from oracle import flow as F

    prob = CASES["owen"]
    sc = Q.Scene(prob)
    W = Q.Warp(F.init_params(3, scale=2.0), rows=1 << 13, uniform_mix=0.1)
    n = 5000
    u = Q.generate_points(prob.generator, 3, 1, n, "f32", seed=prob.seed)
    x, lj = W.forward(u)
    a = sc.accum_buffer("i64")
    la = torch.zeros((n, 5), device="cuda")
    sc.trace_warped(1, n, a, x=x, logj=lj, train_log=la, frac_bits=30)
    b = sc.accum_buffer("i64")
    lb = torch.zeros((n, 5), device="cuda")
    sc.trace_wavefront(1, n, b, sc.wavefront_workspace(n), x=x, logj=lj, train_log=lb, frac_bits=30)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(la, lb)


def test_learned_tracer_on_the_wavefront(Q):
    """The learned tracer's chunked loop gives the same fixed-point image and log with
    the wavefront as with the one-kernel tracer."""
    import torch

    from oracle import flow as F

    prob = CASES["owen"]
    sc = Q.Scene(prob)
    W = Q.Warp(F.init_params(5, scale=2.0), rows=1 << 13, uniform_mix=0.1)
    n = (1 << 13) + 321
    out = []
    for wave in (False, True):
        t = Q.LearnedTracer(sc, W, chunk=1 << 12, wavefront=wave)
        buf = sc.accum_buffer("i64")
        log = torch.zeros((n, 5), device="cuda")
        t.trace(7, n, buf, accum="i64", frac_bits=28, train_log=log)
        out.append((buf, log))
    torch.cuda.synchronize()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
