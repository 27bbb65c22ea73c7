"""The learned warp on the GPU (tensor-core MLPs) against the FP64 oracle with the same
bf16 roundings: the forward warp and its log-Jacobian, the cross-entropy gradient, and
the Adam step.  Remaining differences come from FP32 accumulation order and softmax in
FP32; bin boundaries can flip where u falls within rounding of a cumulative
probability (x stays continuous there, log|J| jumps), so those are counted, not
excluded silently."""
import numpy as np
import pytest

from oracle import flow as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def _params(seed, scale=2.0):
    vec = F.init_params(seed, scale=scale)
    p = F.unpack(vec)
    p["theta0"] = np.random.default_rng(seed + 100).normal(size=F.K_BINS)
    for m in range(2):
        p[f"b{m}0"] = np.random.default_rng(seed + m).normal(size=128) * 0.1
    return F.pack(p)


def test_zero_warp_is_identity(Q):
    import torch

    W = Q.Warp(np.zeros(F.N_PARAMS))
    u = torch.rand((5000, 3), generator=torch.Generator().manual_seed(0)).cuda()
    x, lj = W.forward(u)
    torch.cuda.synchronize()
    assert torch.allclose(x, u, atol=2e-7) and torch.allclose(lj, torch.zeros_like(lj), atol=1e-6)
    assert W.error.item() == 0


@pytest.mark.parametrize("n,mix", [(1000, 0.0), (70001, 0.0), (5000, 0.15)])
def test_forward_matches_oracle(Q, n, mix):
    import torch

    vec = _params(1)
    W = Q.Warp(vec, rows=1 << 15, uniform_mix=mix)
    u = np.random.default_rng(2).uniform(size=(n, 3))
    x, lj = W.forward(torch.tensor(u, dtype=torch.float32).cuda())
    torch.cuda.synchronize()
    xr, ljr = F.warp(u.astype(np.float32).astype(np.float64), vec, use_bf16=True, mix=mix)
    if mix:
        assert lj.max().item() <= -3 * np.log(mix) + 1e-4
    x, lj = x.cpu().numpy(), lj.cpu().numpy()
    # the one-blob inputs are rounded to bf16: a 1e-8 difference in x0 can flip the
    # rounding of a feature (a 2^-8 relative step), which moves x1, x2 by up to ~1e-4
    assert np.abs(x - xr).max() < 1e-3
    assert np.mean(np.abs(x - xr).max(axis=1) < 2e-5) > 0.99
    assert np.mean(np.abs(lj - ljr) < 1e-4) > 0.99
    assert W.error.item() == 0


@pytest.mark.parametrize("mix", [0.0, 0.2])
def test_gradient_matches_oracle(Q, mix):
    import torch

    vec = _params(3, scale=1.5)
    W = Q.Warp(vec, rows=1 << 12, uniform_mix=mix)  # several passes over the samples
    rng = np.random.default_rng(4)
    n = 10000
    x = rng.uniform(size=(n, 3)).astype(np.float32)
    w = rng.uniform(0.0, 2.0, size=n).astype(np.float32)
    loss, g = W.gradient(torch.tensor(x).cuda(), torch.tensor(w).cuda())
    torch.cuda.synchronize()
    lr, gr = F.loss_and_grad(x.astype(np.float64), w.astype(np.float64), vec, use_bf16=True, mix=mix)
    _, gexact = F.loss_and_grad(x.astype(np.float64), w.astype(np.float64), vec, mix=mix)
    g = g.cpu().numpy()
    assert loss.item() == pytest.approx(lr, rel=1e-4)
    assert np.linalg.norm(g - gr) <= 2e-3 * np.linalg.norm(gr)
    assert np.dot(g, gexact) >= 0.99 * np.linalg.norm(g) * np.linalg.norm(gexact)
    for key in ("theta0", "W03", "b13", "W10", "b00"):
        o, sh = F.LAYOUT[key]
        sl = slice(o, o + int(np.prod(sh)))
        assert np.linalg.norm(g[sl] - gr[sl]) <= 5e-3 * np.linalg.norm(gr[sl]) + 1e-9, key
    assert W.error.item() == 0


def test_adam_step_matches_oracle(Q):
    import torch

    vec = _params(5)
    W = Q.Warp(vec)
    rng = np.random.default_rng(6)
    x = rng.uniform(size=(4096, 3)).astype(np.float32)
    w = np.ones(4096, dtype=np.float32)
    m = np.zeros(F.N_PARAMS)
    v = np.zeros(F.N_PARAMS)
    ref = vec.astype(np.float32).astype(np.float64)
    for step in range(1, 4):
        _, g = W.gradient(torch.tensor(x).cuda(), torch.tensor(w).cuda())
        g_host = g.cpu().numpy().astype(np.float64)
        W.adam_step(lr=1e-3)
        ref, m, v = F.adam(ref, g_host, m, v, step, lr=1e-3)
    torch.cuda.synchronize()
    assert np.abs(W.params.cpu().numpy() - ref).max() <= 1e-6
    # the bf16 copies were refreshed from the updated parameters
    o, sh = F.LAYOUT["W00"]
    w00 = W.params[o:o + sh[0] * sh[1]].cpu().bfloat16()
    assert torch.equal(W.wb[:sh[0] * sh[1]].cpu(), w00)


def test_training_moves_the_density_toward_the_samples(Q):
    import torch

    rng = np.random.default_rng(7)
    n = 1 << 16
    x = np.stack([rng.beta(2, 5, n), rng.beta(5, 2, n), rng.beta(2, 2, n)], axis=1).astype(np.float32)
    W = Q.Warp(seed=1, uniform_mix=0.1)
    xs, ws = torch.tensor(x).cuda(), torch.ones(n, device="cuda")
    losses = W.train(xs, ws, epochs=12, batch=1 << 13, lr=1e-2)
    assert losses[-1] < losses[0] - 0.2
    # the trained warp maps uniform points toward the sample distribution: the means of
    # the warped coordinates move from 1/2 toward the beta means 2/7 and 5/7
    u = Q.generate_points("sobol", 3, 1, 1 << 16, "f32")
    xw, lj = W.forward(u)
    mean = xw.mean(0).cpu().numpy()
    assert mean[0] < 0.42 and mean[1] > 0.58, mean
    # unbiased: E_u[|dx/du|] = 1, here a QMC average over a Sobol net; the uniform
    # mixture bounds |dx/du| by 1000, so the average has no heavy tail to chase
    assert torch.exp(lj).mean().item() == pytest.approx(1.0, abs=0.02)
    assert lj.max().item() <= 3 * np.log(10.0) + 1e-4
    assert W.error.item() == 0


def test_fused_forward_agrees_with_the_layer_by_layer_training_forward(Q):
    """The forward pass is one fused tensor-core kernel per conditional; the gradient
    runs the same MLPs layer by layer through the GEMM kernel.  On the forward's own
    samples the training loss with unit weights is -mean log q(x) = mean log |dx/du|,
    so the two paths must agree (a ragged row count exercises the last tile)."""
    import torch

    vec = _params(11)
    W = Q.Warp(vec, rows=1 << 13, uniform_mix=0.05)
    n = (1 << 15) + 77
    u = Q.generate_points("sobol_owen", 3, 1, n, "f32", seed=3)
    x, lj = W.forward(u)
    loss, _ = W.gradient(x, torch.ones(n, device="cuda"))
    torch.cuda.synchronize()
    assert W.error.item() == 0
    assert loss.item() == pytest.approx(lj.double().mean().item(), rel=1e-4, abs=1e-6)
    assert bool(((x >= 0) & (x <= 1)).all())
    assert lj.max().item() <= -3 * np.log(0.05) + 1e-4
