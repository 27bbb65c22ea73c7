"""One trace feeding several observers: each observer's image stack equals the
single-observer trace toward it (bit for bit in fixed point, for single and multiple
scattering, point and finite-star sources), and the FP64 stacks match the oracle run
once per observer."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

pytestmark = pytest.mark.gpu

ANGLES = [(0.0, 0.0), (math.pi / 4, 0.0), (math.pi / 2, 0.3), (2.0, 1.7), (math.pi, 4.0)]


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def _stacks(Q, prob, angles, first, count, fb, precision="f32", half_widths=None, accum="i64"):
    import torch

    sc = Q.Scene(prob)
    dt = torch.int64 if accum == "i64" else torch.float64
    buf = torch.zeros((len(angles), prob.n_images, 3, prob.ny, prob.nx), dtype=dt, device="cuda")
    sc.trace_observers(angles, first, count, buf, half_widths=half_widths, accum=accum, frac_bits=fb,
                       precision=precision)
    torch.cuda.synchronize()
    return buf.cpu()


def _alone(Q, prob, first, count, fb, precision="f32", accum="i64"):
    import torch

    sc = Q.Scene(prob)
    buf = sc.accum_buffer(accum)
    sc.trace(first, count, buf, accum=accum, frac_bits=fb, precision=precision)
    torch.cuda.synchronize()
    return buf[0].cpu()


CASES = {
    "disk_single": S.flared_disk_problem(n=32, nx=40, ny=36),
    "star_single": S.finite_star_disk_problem(n=32, nx=40, ny=36),
    "disk_bilinear": S.flared_disk_problem(n=32, nx=40, ny=36, splat="bilinear"),
    "clumpy_multiple": S.clumpy_problem(n=16, max_orders=6, nx=40, ny=36, per_order=True),
    "clumpy_star_multiple": S.clumpy_problem(n=16, max_orders=4, nx=40, ny=36).replace(
        source="sphere", star_r=0.06, limb_u=0.5),
}


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("name", list(CASES))
def test_each_stack_equals_the_single_observer_trace(Q, name, precision):
    import torch

    prob = CASES[name]
    first, count, fb = 4096, 1 << 13, 36
    hws = [0.8, 1.0, 1.2, 0.9, 1.1]
    got = _stacks(Q, prob, ANGLES, first, count, fb, precision, half_widths=hws)
    for o, (th, ph) in enumerate(ANGLES):
        ref = _alone(Q, prob.replace(theta_obs=th, phi_obs=ph, half_width=hws[o]), first, count, fb, precision)
        assert torch.equal(got[o], ref), (name, o)
    assert bool((got != 0).any())


def test_fp64_stacks_match_the_oracle(Q):
    prob = CASES["star_single"]
    N = 1 << 12
    got = _stacks(Q, prob, ANGLES[:3], 1, N, 0, "f64", accum="f64").numpy()
    for o, (th, ph) in enumerate(ANGLES[:3]):
        ref = O.trace_single(prob.replace(theta_obs=th, phi_obs=ph), 1, N)
        assert np.linalg.norm(got[o, 0] - ref) <= 1e-10 * np.linalg.norm(ref), o
    prob = CASES["clumpy_multiple"]
    got = _stacks(Q, prob, ANGLES[1:3], 1, 2048, 0, "f64", accum="f64").numpy()
    for o, (th, ph) in enumerate(ANGLES[1:3]):
        ref = O.trace_multiple(prob.replace(theta_obs=th, phi_obs=ph), 1, 2048)
        assert np.linalg.norm(got[o] - ref) <= 1e-10 * np.linalg.norm(ref), o


def test_sixteen_observers(Q):
    import torch

    prob = CASES["disk_single"]
    angles = [(math.pi * k / 15, 0.2 * k) for k in range(16)]
    got = _stacks(Q, prob, angles, 1, 1 << 12, 36)
    ref = _alone(Q, prob.replace(theta_obs=angles[15][0], phi_obs=angles[15][1]), 1, 1 << 12, 36)
    assert torch.equal(got[15], ref)
