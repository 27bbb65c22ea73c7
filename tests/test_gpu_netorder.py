"""Net-ordered packet mapping of large blocks: a finite star's further coordinates are
grouped too once a block holds 2^24 points.  The mapping must stay a bijection of each
block: one launch over an aligned 2^24 block gives, in fixed point, the image of two
launches over its 2^23 halves (which keep the three-coordinate order), for both emission
orders, single and multiple scattering, Sobol and Niederreiter."""
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


STAR = S.finite_star_disk_problem(n=256, nx=64, ny=64)  # R* = 6.4 cells: the emission point is ordered
CASES = {
    "inverse": STAR,
    "direct": STAR.replace(emit_order="direct"),
    "niederreiter": STAR.replace(generator="niederreiter"),
    "multiple_direct": STAR.replace(emit_order="direct", max_orders=3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_large_block_order_is_a_bijection(Q, name):
    import torch

    prob = CASES[name]
    n = 1 << 24
    sc = Q.Scene(prob)
    fb = Q.default_frac_bits(prob, n)
    one = sc.accum_buffer("i64")
    sc.trace(n, n, one, frac_bits=fb)
    two = sc.accum_buffer("i64")
    sc.trace(n, n // 2, two, frac_bits=fb)
    sc.trace(n + n // 2, n // 2, two, frac_bits=fb)
    torch.cuda.synchronize()
    assert bool((one != 0).any())
    assert torch.equal(one, two)
