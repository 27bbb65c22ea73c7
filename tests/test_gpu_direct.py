"""Direct light of the source on the GPU against the oracle: point source (one binned
value) and finite limb-darkened star (pixel integrals by subsampling), FP64 and FP32,
through both accumulation modes."""
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


CASES = {
    "point_sphere": S.homogeneous_sphere_problem(sphere_k=0.7, nx=9, ny=9),
    "point_disk_bilinear": S.flared_disk_problem(n=32, nx=17, ny=15, splat="bilinear", theta_obs=1.4),
    "star_disk": S.finite_star_disk_problem(n=32, nx=40, ny=40, half_width=0.08, theta_obs=1.45),
    "star_clumpy": S.clumpy_problem(n=32, max_orders=1, nx=30, ny=30, half_width=0.3).replace(
        source="sphere", star_r=0.2, limb_u=0.3),
}


def _gpu(Q, prob, sub, weight, precision, accum="f64", fb=0):
    import torch

    sc = Q.Scene(prob)
    buf = sc.accum_buffer(accum)
    sc.direct_light(buf, weight=weight, subsamples=sub, accum=accum, frac_bits=fb, precision=precision)
    out = sc.reduce(buf, 1.0, accum=accum, frac_bits=fb)
    torch.cuda.synchronize()
    return out[0].cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_direct_light_matches_oracle(Q, name, precision, tol):
    prob = CASES[name]
    ref = O.direct_light(prob, 5, weight=3.0)
    got = _gpu(Q, prob, 5, 3.0, precision)
    assert ref[0].sum() > 0
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_direct_light_in_fixed_point(Q):
    prob = CASES["star_disk"]
    ref = O.direct_light(prob, 4)
    got = _gpu(Q, prob, 4, 1.0, "f64", accum="i64", fb=50)
    assert np.abs(got - ref).max() <= 2.0 ** -50 * 16 + 1e-15


def test_direct_light_total_of_an_unobscured_star(Q):
    """A star in an empty grid: the pixel integrals add up to 1/(4 pi) up to the
    midpoint rule on the limb."""
    prob = S.Problem(grid=np.zeros((4, 4, 4), np.float32), source="sphere", star_r=0.5, limb_u=0.6, theta_obs=0.9,
                     phi_obs=0.4, half_width=0.6, nx=24, ny=24)
    got = _gpu(Q, prob, 32, 1.0, "f64")
    assert got[0].sum() * 4 * math.pi == pytest.approx(1.0, abs=2e-3)
