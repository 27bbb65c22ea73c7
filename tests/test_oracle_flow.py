"""Pins of the learned-proposal oracle: the warp is a bijection of the unit cube whose
Jacobian integrates to one, q is a normalised density, zero weights give the identity,
the analytic gradient matches finite differences of the loss, and Adam follows its
definition on a quadratic."""
import numpy as np
import pytest

from oracle import flow as F


def test_one_blob_is_gaussian_bumps():
    f = F.one_blob(np.array([0.0, 0.5, 0.99]))
    assert f.shape == (3, F.BLOB)
    centres = (np.arange(F.BLOB) + 0.5) / F.BLOB
    assert np.allclose(f[1], np.exp(-0.5 * ((0.5 - centres) * F.BLOB) ** 2))
    assert np.argmax(f[2]) == F.BLOB - 1


def test_zero_network_is_the_identity():
    vec = np.zeros(F.N_PARAMS)
    u = np.random.default_rng(0).uniform(size=(500, 3))
    x, logj = F.warp(u, vec)
    assert np.allclose(x, u, atol=1e-15) and np.allclose(logj, 0.0, atol=1e-15)


def test_warp_is_a_bijection_with_unit_jacobian_mass():
    vec = F.init_params(3, scale=3.0)
    p = F.unpack(vec)
    p["theta0"] = np.random.default_rng(1).normal(size=F.K_BINS)
    vec = F.pack(p)
    rng = np.random.default_rng(2)
    u = rng.uniform(size=(4000, 3))
    x, logj = F.warp(u, vec)
    assert np.all((x >= 0) & (x <= 1))
    # inverse: u_l = F_l(x_l | x_<l) with the conditionals at the final coordinates
    Q0, Q1, Q2 = F.conditionals(x, vec)
    for l, Q in enumerate((Q0, Q1, Q2)):
        assert np.allclose(F.cdf(x[:, l], Q), u[:, l], atol=1e-12)
    # log |dx/du| = -log q(x)
    assert np.allclose(logj, -F.log_density(x, vec), atol=1e-12)
    # E_u[|dx/du|] = volume of the cube = 1 (midpoint grid over u, exact up to the grid)
    g = (np.arange(24) + 0.5) / 24
    U = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    _, lj = F.warp(U, vec)
    assert np.exp(lj).mean() == pytest.approx(1.0, abs=2e-2)


def test_density_integrates_to_one_exactly():
    """q is piecewise constant in x on a 32^3 lattice only for x0; numerically integrate
    over a midpoint grid fine enough for the one-blob smoothness of the conditionals."""
    vec = F.init_params(4, scale=2.0)
    n = 48
    g = (np.arange(n) + 0.5) / n
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    q = np.exp(F.log_density(X, vec))
    assert q.mean() == pytest.approx(1.0, abs=3e-2)
    # conditional normalisation is exact: for each (x0, x1) the x2 marginal sums to one
    Q0, Q1, Q2 = F.conditionals(X[:100], vec)
    assert np.allclose(Q2.sum(axis=1), 1.0) and np.allclose(Q1.sum(axis=1), 1.0)


@pytest.mark.parametrize("use_bf16,mix", [(False, 0.0), (True, 0.0), (False, 0.2)])
def test_gradient_matches_finite_differences(use_bf16, mix):
    rng = np.random.default_rng(5)
    vec = F.init_params(6, scale=1.5)
    x = rng.uniform(size=(64, 3))
    w = rng.uniform(0.1, 2.0, size=64)
    loss, g = F.loss_and_grad(x, w, vec, mix=mix)
    idx = rng.choice(F.N_PARAMS, size=40, replace=False)
    idx = np.concatenate([idx, [0, 5, F.LAYOUT["b03"][0], F.LAYOUT["W13"][0] + 7]])
    for i in idx:
        h = 1e-6
        e = np.zeros(F.N_PARAMS)
        e[i] = h
        fd = (F.loss_and_grad(x, w, vec + e, mix=mix)[0] - F.loss_and_grad(x, w, vec - e, mix=mix)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    if use_bf16:
        lb, gb = F.loss_and_grad(x, w, vec, use_bf16=True)
        assert lb == pytest.approx(loss, rel=2e-2)
        assert np.dot(gb, g) > 0.9 * np.linalg.norm(gb) * np.linalg.norm(g)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(0).normal(size=1000) * 10 ** np.random.default_rng(1).uniform(-5, 5, size=1000)
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(F.bf16(a), ref)


def test_training_reduces_the_loss_toward_a_known_density():
    """Samples of a separable target density: minimising the cross-entropy must move
    q toward it (loss decreases and approaches the target's entropy bound)."""
    rng = np.random.default_rng(7)
    n = 4096
    x = np.stack([rng.beta(2, 5, n), rng.beta(5, 2, n), rng.uniform(size=n)], axis=1)
    w = np.ones(n)
    vec = F.init_params(8)
    m = np.zeros_like(vec)
    v = np.zeros_like(vec)
    l0 = F.loss_and_grad(x, w, vec)[0]
    for step in range(1, 61):
        loss, g = F.loss_and_grad(x, w, vec)
        vec, m, v = F.adam(vec, g, m, v, step, lr=3e-3)
    assert loss < l0 - 0.15  # two beta marginals have entropy well below 0 (uniform)


def test_adam_definition_on_a_quadratic():
    vec = np.array([1.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    new, m, v = F.adam(vec, 2 * vec, m, v, 1, lr=0.1)
    assert np.allclose(new, vec - 0.1 * np.sign(vec))  # first step: m_hat/sqrt(v_hat) = sign(g)


def test_uniform_mixture_bounds_the_jacobian_and_stays_a_bijection():
    """With bin masses (1 - mix) softmax + mix / 32 every conditional density is at
    least mix, so |dx/du| <= mix^-3, even for a sharply peaked network; the warp
    still inverts through the CDFs and log |dx/du| = -log q(x)."""
    mix = 0.1
    vec = F.init_params(9, scale=8.0)
    p = F.unpack(vec)
    p["theta0"] = np.zeros(F.K_BINS)
    p["theta0"][3] = 40.0  # almost all of x0's mass in one bin without the mixture
    vec = F.pack(p)
    u = np.random.default_rng(10).uniform(size=(3000, 3))
    x, logj = F.warp(u, vec, mix=mix)
    assert np.all(logj <= -3 * np.log(mix) + 1e-12)
    # without the mixture 1 / q is huge outside the peak (x0 in another bin)
    assert (-F.log_density(u, vec)).max() > -3 * np.log(mix) + 10.0
    assert (-F.log_density(u, vec, mix=mix)).max() <= -3 * np.log(mix) + 1e-12
    for l, Q in enumerate(F.conditionals(x, vec, mix=mix)):
        assert np.allclose(Q.sum(axis=1), 1.0)
        assert Q.min() >= mix / F.K_BINS * (1 - 1e-12)
        assert np.allclose(F.cdf(x[:, l], Q), u[:, l], atol=1e-12)
    assert np.allclose(logj, -F.log_density(x, vec, mix=mix), atol=1e-12)
