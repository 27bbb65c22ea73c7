"""FP64 oracle of the learned proposal: a piecewise-linear autoregressive warp of the
first-scattering coordinates (u0, u1, u2) -> (x0, x1, x2) of the unit cube, trained by
minimising the cross-entropy -E[w log q(x)] of logged packets (Mueller et al., "Neural
Importance Sampling", ACM TOG 2019, piecewise-linear coupling, written here in the
autoregressive form: every conditional reads final coordinates, so log q needs no
inverse pass).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark baseline).  Plain numpy, one
operation per line of the definition:

  x0 ~ pdf K Q0[b] on bin b = floor(K x0),  Q0 = softmax(theta0)
  x1 ~ pdf K Q1[b],  Q1 = softmax(MLP1(onehot(x0)))
  x2 ~ pdf K Q2[b],  Q2 = softmax(MLP2(onehot(x0), onehot(x1)))
  q(x) = prod_l K Q_l[b_l];  sampling x_l = F_l^-1(u_l), |dx/du| = 1 / q(x)
  MLP: 4 layers, ReLU, width 128, input padded to 128 features.
The estimator of an integral over the cube stays unbiased: f(x(u)) |dx/du|.
With bf16=True the weights, the input features and the hidden activations are rounded
to bfloat16 where the GPU stores them (accumulation stays exact here).
"""
from __future__ import annotations

import numpy as np

K_BINS = 32
BLOB = 32
WIDTH = 128
IN = 128
LAYERS = [(WIDTH, IN), (WIDTH, WIDTH), (WIDTH, WIDTH), (K_BINS, WIDTH)]  # (out, in)


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def param_layout():
    """Offsets of the FP32 parameter vector: theta0, then for each MLP and layer W then b."""
    off, out = 0, {"theta0": (0, (K_BINS,))}
    off = K_BINS
    for m in range(2):
        for l, (o, i) in enumerate(LAYERS):
            out[f"W{m}{l}"] = (off, (o, i))
            off += o * i
            out[f"b{m}{l}"] = (off, (o,))
            off += o
    return out, off


LAYOUT, N_PARAMS = param_layout()


def unpack(vec):
    return {k: np.asarray(vec[o:o + int(np.prod(s))], dtype=np.float64).reshape(s) for k, (o, s) in LAYOUT.items()}


def pack(params) -> np.ndarray:
    v = np.zeros(N_PARAMS)
    for k, (o, s) in LAYOUT.items():
        v[o:o + int(np.prod(s))] = np.asarray(params[k]).ravel()
    return v


def init_params(seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """He-style random weights, zero biases, zero theta0 (uniform x0); the output layer
    starts small so the initial warp is close to the identity."""
    rng = np.random.default_rng(seed)
    p = {"theta0": np.zeros(K_BINS)}
    for m in range(2):
        for l, (o, i) in enumerate(LAYERS):
            std = scale * np.sqrt(2.0 / i) * (0.1 if l == 3 else 1.0)
            p[f"W{m}{l}"] = rng.standard_normal((o, i)) * std
            p[f"b{m}{l}"] = np.zeros(o)
    return pack(p)


def one_blob(v, n=BLOB):
    """One-blob encoding: Gaussian bumps (sigma = 1/n) at the bin centres."""
    centres = (np.arange(n) + 0.5) / n
    return np.exp(-0.5 * ((np.asarray(v)[:, None] - centres[None, :]) * n) ** 2)


def features(x, m, use_bf16=False):
    """Input of MLP m (m = 0 conditions x1 on x0, m = 1 conditions x2 on x0, x1)."""
    B = x.shape[0]
    f = np.zeros((B, IN))
    f[:, 0:BLOB] = one_blob(x[:, 0])
    if m == 1:
        f[:, BLOB:2 * BLOB] = one_blob(x[:, 1])
    return bf16(f) if use_bf16 else f


def mlp(f, p, m, use_bf16=False):
    """Logits [B][K_BINS] and the hidden activations (pre-activation kept for backprop)."""
    h = f
    cache = [h]
    for l in range(4):
        W, b = p[f"W{m}{l}"], p[f"b{m}{l}"]
        if use_bf16:
            W = bf16(W)
        z = h @ W.T + b
        if l < 3:
            h = np.maximum(z, 0.0)
            if use_bf16:
                h = bf16(h)
            cache.append(h)
        else:
            h = z
    return h, cache


def softmax(z):
    z = z - z.max(axis=-1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=-1, keepdims=True)


def mixture(S, mix):
    """Defensive mixture with the uniform bin masses: (1 - mix) S + mix / K, so that
    K Q >= mix and |dx/du| = 1 / q(x) <= mix^-3."""
    return (1.0 - mix) * S + mix / K_BINS


def inverse_cdf(u, Q):
    """x with F(x) = u for the piecewise-constant pdf K Q[b] on K equal bins; returns x, b."""
    c = np.concatenate([np.zeros((Q.shape[0], 1)), np.cumsum(Q, axis=1)], axis=1)
    b = np.array([min(max(np.searchsorted(c[j], u[j], side="right") - 1, 0), K_BINS - 1) for j in range(len(u))])
    rows = np.arange(len(u))
    x = (b + (u - c[rows, b]) / Q[rows, b]) / K_BINS
    return np.clip(x, 0.0, 1.0), b


def cdf(x, Q):
    b = np.minimum((x * K_BINS).astype(int), K_BINS - 1)
    c = np.concatenate([np.zeros((Q.shape[0], 1)), np.cumsum(Q, axis=1)], axis=1)
    rows = np.arange(len(x))
    return c[rows, b] + (x * K_BINS - b) * Q[rows, b]


def conditionals(x, vec, use_bf16=False, mix=0.0):
    """Q0 (one row per sample), Q1, Q2 at the coordinates x [B][3]."""
    p = unpack(vec)
    B = x.shape[0]
    Q0 = np.repeat(mixture(softmax(p["theta0"]), mix)[None, :], B, axis=0)
    L1, _ = mlp(features(x, 0, use_bf16), p, 0, use_bf16)
    L2, _ = mlp(features(x, 1, use_bf16), p, 1, use_bf16)
    return Q0, mixture(softmax(L1), mix), mixture(softmax(L2), mix)


def warp(u, vec, use_bf16=False, mix=0.0):
    """x = T(u) and log |dx/du| (= -log q(x)) for points u [B][3]."""
    p = unpack(vec)
    B = u.shape[0]
    x = np.zeros((B, 3))
    logq = np.zeros(B)
    Q0 = np.repeat(mixture(softmax(p["theta0"]), mix)[None, :], B, axis=0)
    x[:, 0], b = inverse_cdf(u[:, 0], Q0)
    logq += np.log(K_BINS * Q0[np.arange(B), b])
    L1, _ = mlp(features(x, 0, use_bf16), p, 0, use_bf16)
    Q1 = mixture(softmax(L1), mix)
    x[:, 1], b = inverse_cdf(u[:, 1], Q1)
    logq += np.log(K_BINS * Q1[np.arange(B), b])
    L2, _ = mlp(features(x, 1, use_bf16), p, 1, use_bf16)
    Q2 = mixture(softmax(L2), mix)
    x[:, 2], b = inverse_cdf(u[:, 2], Q2)
    logq += np.log(K_BINS * Q2[np.arange(B), b])
    return x, -logq


def log_density(x, vec, use_bf16=False, mix=0.0):
    Qs = conditionals(x, vec, use_bf16, mix)
    rows = np.arange(x.shape[0])
    out = np.zeros(x.shape[0])
    for l, Q in enumerate(Qs):
        b = np.minimum((x[:, l] * K_BINS).astype(int), K_BINS - 1)
        out += np.log(K_BINS * Q[rows, b])
    return out


def loss_and_grad(x, w, vec, use_bf16=False, mix=0.0):
    """loss = -sum_j w_j log q(x_j) / sum_j w_j and its gradient w.r.t. the parameters.
    With the mixture Q = (1 - mix) S + mix / K (S = softmax(z)) the derivative of
    log Q_b by the logits is r (e_b - S), r = (1 - mix) S_b / Q_b."""
    p = unpack(vec)
    B = x.shape[0]
    rows = np.arange(B)
    W = w.sum()
    g = {k: np.zeros(s) for k, (o, s) in LAYOUT.items()}
    loss = 0.0
    # x0: unconditional logits
    S0 = softmax(p["theta0"])
    Q0 = mixture(S0, mix)
    b0 = np.minimum((x[:, 0] * K_BINS).astype(int), K_BINS - 1)
    loss -= np.sum(w * np.log(K_BINS * Q0[b0])) / W
    onehot0 = np.zeros((B, K_BINS))
    onehot0[rows, b0] = 1.0
    r0 = (1.0 - mix) * S0[b0] / Q0[b0]
    g["theta0"] = -((w / W * r0)[:, None] * (onehot0 - S0[None, :])).sum(axis=0)
    for m in range(2):
        L, cache = mlp(features(x, m, use_bf16), p, m, use_bf16)
        Sm = softmax(L)
        Q = mixture(Sm, mix)
        bl = np.minimum((x[:, m + 1] * K_BINS).astype(int), K_BINS - 1)
        loss -= np.sum(w * np.log(K_BINS * Q[rows, bl])) / W
        oh = np.zeros((B, K_BINS))
        oh[rows, bl] = 1.0
        r = (1.0 - mix) * Sm[rows, bl] / Q[rows, bl]
        d = -(w / W * r)[:, None] * (oh - Sm)  # d loss / d logits
        for l in (3, 2, 1, 0):
            h_in = cache[l]
            Wl = p[f"W{m}{l}"]
            if use_bf16:  # the GPU stores the backward signal and the weights in bf16
                Wl = bf16(Wl)
                d = bf16(d)
            g[f"W{m}{l}"] = d.T @ h_in
            g[f"b{m}{l}"] = d.sum(axis=0)
            if l > 0:
                d = (d @ Wl) * (cache[l] > 0)
    return loss, pack(g)


def adam(vec, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; returns new (vec, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return vec - lr * mh / (np.sqrt(vh) + eps), m, v
