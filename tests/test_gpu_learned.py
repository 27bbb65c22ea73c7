"""The learned proposal inside the multiple-scattering tracer: the warped FP64 trace
against the oracle fed the same warped coordinates and Jacobians, the per-packet
training log, the plain path through the same entry point, and unbiasedness of the
learned estimator against plain QMC after training on the tracer's own log."""
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


def _problem(n=16, **kw):
    return S.clumpy_problem(n=n, max_orders=8, nx=48, ny=40, half_width=0.9, **kw)


def _warp_params(seed=3):
    from oracle import flow as F

    vec = F.init_params(seed, scale=2.0)
    p = F.unpack(vec)
    p["theta0"] = np.random.default_rng(seed).normal(size=F.K_BINS)
    return F.pack(p)


def _warp(Q, mix=0.1, seed=3):
    return Q.Warp(_warp_params(seed), rows=1 << 14, uniform_mix=mix)


@pytest.mark.parametrize("first,count", [(1, 3000), (4096, 1 << 13)])
def test_warped_fp64_trace_matches_oracle(Q, first, count):
    import torch

    prob = _problem()
    sc = Q.Scene(prob)
    W = _warp(Q)
    tr = Q.LearnedTracer(sc, W, chunk=1 << 12)  # several chunks
    buf = sc.accum_buffer("f64")
    log = torch.zeros((count, 5), dtype=torch.float32, device="cuda")
    tr.trace(first, count, buf, frac_bits=0, accum="f64", precision="f64", train_log=log)
    u = Q.generate_points(prob.generator, 3, first, count, "f32")
    x, lj = W.forward(u)
    torch.cuda.synchronize()
    assert W.error.item() == 0
    xh = x.cpu().numpy().astype(np.float64)
    ljh = lj.cpu().numpy().astype(np.float64)
    ref, rlog = O.trace_multiple_warped(prob, first, count, xh, ljh, train_log=True)
    got = buf[0].cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    lg = log.cpu().numpy()
    assert np.array_equal(lg[:, :3], x.cpu().numpy())
    assert np.allclose(lg[:, 3:], rlog[:, 3:], rtol=1e-6, atol=1e-30)
    # the warp moved the points, and the weights are bounded by mix^-3
    assert np.abs(xh - u.cpu().numpy()).max() > 0.05
    assert ljh.max() <= 3 * np.log(10.0) + 1e-4


def test_learned_chain_end_to_end_against_the_oracle_alone(Q):
    """The whole learned chain on each side with nothing shared: the GPU generates the
    float points, warps them on the tensor cores (qmcrt_warp_forward, bf16) and traces
    them (FP64 trace, FP64 image); the oracle takes the same float points through its
    own flow with the same bf16 roundings (oracle/flow.py) and its own warped trace.

    Tolerance, from the flips counted: a point whose GPU x differs from the oracle's by
    more than the forward's float rounding (2e-5, or 1e-4 in log J) took another
    bf16 rounding of a feature and can move its whole contribution, so the flipped
    packets' logged intensities (both sides) enter the L1 budget in full; the others
    move their contributions by their coordinate change, ~2e-5 x (about 30 pixels per
    unit of sky for the tent splat) ~ 1e-3 of their own intensity at most."""
    import torch

    from oracle import flow as F

    prob = _problem().replace(splat="bilinear")
    sc = Q.Scene(prob)
    vec = _warp_params()
    W = Q.Warp(vec, rows=1 << 14, uniform_mix=0.1)
    first, count = 1, 1 << 13
    buf = sc.accum_buffer("f64")
    log = torch.zeros((count, 5), dtype=torch.float32, device="cuda")
    Q.LearnedTracer(sc, W, chunk=1 << 12).trace(first, count, buf, accum="f64", precision="f64", train_log=log)
    torch.cuda.synchronize()
    assert W.error.item() == 0
    got, glog = buf[0].cpu().numpy(), log.cpu().numpy().astype(np.float64)

    u = O.generate_points(prob.generator, 3, first, count, "f32").astype(np.float64)
    xr, ljr = F.warp(u, vec, use_bf16=True, mix=0.1)
    ref, rlog = O.trace_multiple_warped(prob, first, count, xr, ljr, train_log=True)

    flipped = np.abs(glog[:, :3] - xr).max(axis=1) > 2e-5
    assert flipped.mean() <= 0.02, flipped.mean()
    total = rlog[:, 3].sum()
    budget = (rlog[flipped, 3].sum() + glog[flipped, 3].sum() + 1e-3 * rlog[~flipped, 3].sum()) / total
    err_l1 = np.abs(got[0] - ref[0]).sum() / np.abs(ref[0]).sum()
    assert err_l1 <= budget, (err_l1, budget, flipped.sum())
    # the flips are rare enough that the end-to-end image is close in L2 as well
    assert np.linalg.norm(got - ref) <= 0.05 * np.linalg.norm(ref)


def test_plain_entry_point_is_the_multiple_tracer_and_logs(Q):
    import torch

    prob = _problem()
    sc = Q.Scene(prob)
    count, fb = 1 << 13, 40
    a = sc.accum_buffer("i64")
    sc.trace(1, count, a, frac_bits=fb, precision="f64")
    b = sc.accum_buffer("i64")
    log = torch.zeros((count, 5), dtype=torch.float32, device="cuda")
    Q.LearnedTracer(sc, None).trace(1, count, b, frac_bits=fb, accum="i64", precision="f64", train_log=log)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    _, rlog = O.trace_multiple_warped(prob, 1, count, train_log=True)
    lg = log.cpu().numpy()
    assert np.array_equal(lg[:, :3], rlog[:, :3].astype(np.float32))
    assert np.allclose(lg[:, 3:], rlog[:, 3:], rtol=1e-6, atol=1e-30)


def test_fp32_warped_trace_is_close_to_fp64(Q):
    import torch

    prob = _problem(n=32)
    sc = Q.Scene(prob)
    tr = Q.LearnedTracer(sc, _warp(Q))
    count = 1 << 16
    fb = Q.default_frac_bits(prob, count, tr.weight_bound())
    imgs = []
    for prec in ("f32", "f64"):
        buf = sc.accum_buffer("i64")
        tr.trace(1, count, buf, frac_bits=fb, accum="i64", precision=prec)
        imgs.append(sc.reduce(buf, 1.0 / count, frac_bits=fb)[0].cpu().numpy())
    torch.cuda.synchronize()
    assert np.linalg.norm(imgs[0] - imgs[1]) <= 5e-3 * np.linalg.norm(imgs[1])


def test_unbounded_warp_refuses_fixed_point(Q):
    prob = _problem()
    sc = Q.Scene(prob)
    tr = Q.LearnedTracer(sc, _warp(Q, mix=0.0))
    with pytest.raises(Q.QmcrtError):
        tr.trace(1, 128, sc.accum_buffer("i64"), frac_bits=10, accum="i64")


def test_warp_rejects_sphere_source_and_half_given_warp(Q):
    import torch

    prob = S.flared_disk_problem(n=16, nx=16, ny=16, source="sphere", star_r=0.05, max_orders=3)
    sc = Q.Scene(prob)
    x = torch.zeros((128, 3), device="cuda")
    lj = torch.zeros(128, device="cuda")
    with pytest.raises(Q.QmcrtError):
        sc.trace_warped(1, 128, sc.accum_buffer("i64"), x=x, logj=lj)
    sc2 = Q.Scene(_problem())
    with pytest.raises(Q.QmcrtError):
        sc2.trace_warped(1, 128, sc2.accum_buffer("i64"), x=x)


def test_learned_estimator_is_unbiased_after_training(Q):
    """Train the warp on the tracer's own log of plain packets, then trace with it
    on independently Owen-scrambled point sets: the mean total flux over the replicates
    agrees with a plain image of 64x the packets within four standard errors, and the
    per-pixel error is no worse than plain QMC's at the same count."""
    import torch

    prob = _problem(n=32)
    sc = Q.Scene(prob)
    n_log = 1 << 18
    log = torch.zeros((n_log, 5), dtype=torch.float32, device="cuda")
    plain = Q.LearnedTracer(sc, None)
    plain.trace(1, n_log, sc.accum_buffer("f64"), train_log=log)
    W = Q.Warp(seed=2, uniform_mix=0.1)
    losses = W.train(log[:, :3].contiguous(), log[:, 3].contiguous(), epochs=6, batch=1 << 14, lr=3e-3)
    assert np.mean(losses[-4:]) < losses[0] - 0.05

    def image(s, tracer, first, count):
        buf = s.accum_buffer("f64")
        tracer.trace(first, count, buf)
        return s.reduce(buf, 1.0 / count, accum="f64")[0, 0].cpu().numpy()

    N = 1 << 16
    ref = image(sc, plain, 1 << 22, 1 << 22)
    tot, e_l, e_p = [], [], []
    for seed in range(1, 9):
        s = Q.Scene(prob.replace(generator="sobol_owen", seed=seed), grid_device=sc.grid)
        b = image(s, Q.LearnedTracer(s, W), 1, N)
        a = image(s, Q.LearnedTracer(s, None), 1, N)
        tot.append(b.sum() / ref.sum() - 1)
        e_l.append(np.linalg.norm(b - ref) / np.linalg.norm(ref))
        e_p.append(np.linalg.norm(a - ref) / np.linalg.norm(ref))
    torch.cuda.synchronize()
    assert W.error.item() == 0
    tot = np.array(tot)
    se = tot.std(ddof=1) / np.sqrt(len(tot))
    assert abs(tot.mean()) < 4 * se + 2e-3, (tot.mean(), se)
    assert np.mean(e_l) < 1.1 * np.mean(e_p), (np.mean(e_l), np.mean(e_p))
