"""Parity at the benchmark's full sizes and launch configurations, on outputs the oracle
can compute one packet at a time:

* single scattering: one step of the benchmark (2^26 packets of the 256^3 disk, one
  aligned block of the sequence, FP32 trace, fixed-point image) -- sampled packets of the
  packet log against the oracle, and the image total against the log;
* multiple scattering: the clumpy workload at 2^24 packets through the wavefront (the
  bench's path for it) -- sampled packets of the training log (sum of each packet's
  in-image intensities over all orders) against the oracle, and the image total against
  the log."""
import numpy as np
import pytest

from fp32_check import fp32_packet_check
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


def _close_fraction(got, ref, rtol):
    """Fraction of packets within rtol of the oracle, relative to max(|ref|, mean |ref|)."""
    scale = np.maximum(np.abs(ref), np.abs(ref).mean() + 1e-300)
    return float(np.mean(np.abs(got - ref) <= rtol * scale))


def test_benchmark_step_single_scattering_sampled(Q):
    import torch

    prob = S.flared_disk_problem(n=256)
    n = 1 << 26
    first = n  # the benchmark's first step: indices 2^26 .. 2^27 - 1
    sc = Q.Scene(prob)
    fb = Q.default_frac_bits(prob, n)
    buf = sc.accum_buffer("i64")
    lg = torch.zeros((n, 9), dtype=torch.float64, device="cuda")
    sc.trace(first, n, buf, frac_bits=fb, log=lg)
    img = sc.reduce(buf, 1.0, frac_bits=fb)[0, 0]
    starts = np.unique(np.random.default_rng(7).integers(0, n - 100, 30))  # 30 runs of 100 packets
    sample = (starts[:, None] + np.arange(100)[None, :]).ravel()
    got = lg[torch.as_tensor(sample, device="cuda")].cpu().numpy()
    ref = np.concatenate([O.trace_single(prob, first + int(j0), 100, log=True)[1] for j0 in starts])
    assert np.array_equal(got[:, 8], ref[:, 8])  # status: contributed, tau_1 < tau_min, occulted
    # I, Q, U and sky position within 1e-5 of the packet's own I on the well-conditioned
    # packets (all of them in practice), the ill-conditioned ones bounded separately
    fp32_packet_check(prob, first + sample, got, ref)
    # the image holds exactly the logged in-frame intensities
    ok = (lg[:, 8] == 0) & (lg[:, 6].abs() < prob.half_width) & (lg[:, 7].abs() < prob.half_width)
    assert float(img.sum()) == pytest.approx(float(lg[ok, 3].sum()), rel=1e-9)


def test_benchmark_multiple_scattering_wavefront_sampled(Q):
    import torch

    prob = S.clumpy_problem(n=128)
    n = 1 << 24
    sc = Q.Scene(prob)
    fb = Q.default_frac_bits(prob, n)
    buf = sc.accum_buffer("i64")
    log = torch.zeros((n, 5), dtype=torch.float32, device="cuda")
    sc.trace_wavefront(n, n, buf, sc.wavefront_workspace(n), frac_bits=fb, train_log=log)
    img = sc.reduce(buf, 1.0, frac_bits=fb)[0, 0]
    starts = np.unique(np.random.default_rng(11).integers(0, n - 100, 15))  # 15 runs of 100 packets
    sample = (starts[:, None] + np.arange(100)[None, :]).ravel()
    got = log[torch.as_tensor(sample, device="cuda")].cpu().numpy().astype(np.float64)
    ref = np.concatenate([O.trace_multiple_warped(prob, n + int(j0), 100, train_log=True)[1] for j0 in starts])
    # first-order u: the FP32 value of a point is its FP64 value rounded toward zero
    f = ref[:, :3].astype(np.float32)
    f = np.where(f.astype(np.float64) > ref[:, :3], np.nextafter(f, np.float32(0)), f)
    assert np.array_equal(got[:, :3], f.astype(np.float64))
    assert _close_fraction(got[:, 3], ref[:, 3], 1e-4) >= 0.99  # sum of in-image I over all orders
    assert _close_fraction(got[:, 3], ref[:, 3], 1e-2) == 1.0
    # the image's I total is the logged sum over all packets (FP32 per packet, FP64 image)
    assert float(img.sum()) == pytest.approx(float(log[:, 3].double().sum()), rel=1e-5)
