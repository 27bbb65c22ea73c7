"""GPU point sets through the C ABI, bit-exact against the CPU oracle (Sec. 3.1)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def _gpu(Q, kind, dims, first, count, fmt, seed=0, total_n=0):
    import torch

    out = Q.generate_points(kind, dims, first, count, fmt, seed=seed, total_n=total_n)
    torch.cuda.synchronize()
    a = out.cpu().numpy()
    return a.view(np.uint32) if fmt == "u32" else a


CASES = [
    ("sobol", 5, 1, 1000, 0, 0), ("sobol", 80, 123_457, 777, 0, 0), ("sobol", 256, 1, 300, 0, 0),
    ("sobol_owen", 5, 1, 1000, 7, 0), ("sobol_owen", 80, 99, 513, 2 ** 40 + 3, 0),
    ("halton", 5, 1, 1000, 0, 0), ("halton", 80, 4_000_000_000, 257, 0, 0),
    ("hammersley", 5, 1, 1000, 0, 1000), ("hammersley", 3, 5, 95, 0, 99),
    ("philox", 5, 1, 1000, 12345, 0), ("philox", 9, 2 ** 33 + 1, 100, 2 ** 63 + 5, 0),
    ("niederreiter", 5, 1, 1000, 0, 0), ("niederreiter", 256, 2 ** 31 + 7, 300, 0, 0),
    ("faure", 3, 1, 1000, 0, 0), ("faure", 5, 3_000_000_000, 257, 0, 0), ("faure", 80, 1, 700, 0, 0),
]


@pytest.mark.parametrize("kind,dims,first,count,seed,total_n", CASES)
@pytest.mark.parametrize("fmt", ["u32", "f32", "f64"])
def test_points_bit_exact(Q, kind, dims, first, count, seed, total_n, fmt):
    if fmt == "u32" and kind in ("halton", "hammersley", "faure"):
        pytest.skip("no integer form")
    got = _gpu(Q, kind, dims, first, count, fmt, seed, total_n)
    ref = O.generate_points(kind, dims, first, count, fmt, seed=seed, total_n=total_n)
    assert got.shape == ref.shape
    assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))


def test_points_large_block_sampled(Q):
    """Full-size block (2^24 x 3, the single-scattering workload's point set): sampled
    rows against the oracle, plus exact stratification of the first 2^20 rows."""
    n = 1 << 24
    got = _gpu(Q, "sobol", 3, 1, n, "u32")
    rng = np.random.default_rng(0)
    rows = np.unique(rng.integers(0, n, 4096))
    for r in rows[:512]:
        assert np.array_equal(got[r], O.generate_points("sobol", 3, 1 + int(r), 1, "u32")[0])
    # indices 1..2^20 plus the point 0 form a (0, 20, 1)-net in each dimension
    head = np.concatenate([np.zeros((1, 3), np.uint32), got[: (1 << 20) - 1]])
    for d in range(3):
        assert len(np.unique(head[:, d] >> 12)) == 1 << 20


def test_points_empty_and_single(Q):
    import torch

    out = torch.full((1, 3), -1.0, dtype=torch.float64, device="cuda")
    Q.qmcrt_generate_points(Q.points_desc("sobol", 3, 1, 0), out.data_ptr())
    torch.cuda.synchronize()
    assert torch.all(out == -1.0)
    got = _gpu(Q, "sobol", 3, 1, 1, "f64")
    assert np.array_equal(got, [[0.5, 0.5, 0.5]])
