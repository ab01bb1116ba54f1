"""FP64 oracle of the learned-proposal network (test infrastructure only).

x (3z neighbour spin components) -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> o = W3 h2 + b3;
mu = o[:3] / |o[:3]|, kappa = softplus(o[3]) + 1e-4; the loss is the negative
log-likelihood of the site spin y under the 3D von Mises-Fisher law with density
kappa / (4 pi sinh kappa) * exp(kappa mu . y).  Parameters use the packed layout
[W1 H*nin][b1 H][W2 H*H][b2 H][W3 4*H][b3 4] of the C ABI.  The gradient is pinned
against finite differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

H = 64


def unpack(p, nin):
    p = np.asarray(p, np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, nin)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (4, H)), ("b3", (4,))):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def n_params(nin):
    return H * nin + H + H * H + H + 4 * H + 4


def forward(p, x, nin):
    w = unpack(p, nin)
    x = np.asarray(x, np.float64)
    h1 = np.tanh(x @ w["W1"].T + w["b1"])
    h2 = np.tanh(h1 @ w["W2"].T + w["b2"])
    o = h2 @ w["W3"].T + w["b3"]
    vn = np.linalg.norm(o[:, :3], axis=1)
    mu = o[:, :3] / vn[:, None]
    kappa = np.logaddexp(0.0, o[:, 3]) + 1e-4
    return mu, kappa, (x, h1, h2, o, vn)


def nll(p, x, y, nin):
    """Sum over samples of -log q(y | x) for the vMF law."""
    mu, k, _ = forward(p, x, nin)
    y = np.asarray(y, np.float64)
    log_norm = np.log(k) - np.log(4 * np.pi) - (k + np.log1p(-np.exp(-2 * k)) - np.log(2.0))
    return float(-(log_norm + k * (mu * y).sum(1)).sum())


def grad(p, x, y, nin):
    """Gradient of nll by explicit back-propagation (FP64)."""
    w = unpack(p, nin)
    mu, k, (x, h1, h2, o, vn) = forward(p, x, nin)
    y = np.asarray(y, np.float64)
    muy = (mu * y).sum(1)
    dk = 1.0 / np.tanh(k) - 1.0 / k - muy
    dO = np.zeros_like(o)
    dO[:, 3] = dk / (1.0 + np.exp(-o[:, 3]))
    dO[:, :3] = -k[:, None] * (y - mu * muy[:, None]) / vn[:, None]
    d2 = (dO @ w["W3"]) * (1 - h2 ** 2)
    d1 = (d2 @ w["W2"]) * (1 - h1 ** 2)
    g = {"W3": dO.T @ h2, "b3": dO.sum(0), "W2": d2.T @ h1, "b2": d2.sum(0),
         "W1": d1.T @ x, "b1": d1.sum(0)}
    return np.concatenate([g[n].ravel() for n in ("W1", "b1", "W2", "b2", "W3", "b3")])


def init(nin, seed):
    """Glorot-uniform weights, zero biases (the same recipe the tests use on the GPU)."""
    g = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((H, nin), (H, H), (4, H)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(g.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)
