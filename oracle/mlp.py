"""FP64 oracle of the learned-proposal network (test infrastructure only).

x (3z neighbour spin components) -> h1 = tanh(W1 x + b1) -> h2 = tanh(W2 h1 + b2)
[-> h3 = tanh(Wm h2 + bm) with three hidden layers] -> o = W3 h_last + b3;
mu = o[:3] / |o[:3]|, kappa = softplus(o[3]) + 1e-4; the loss is the negative
log-likelihood of the site spin y under the 3D von Mises-Fisher law with density
kappa / (4 pi sinh kappa) * exp(kappa mu . y).  Parameters use the packed layout
[W1 H*nin][b1 H][W2 H*H][b2 H]([Wm H*H][bm H])[W3 4*H][b3 4] of the C ABI, `depth`
being the number of hidden layers (2 or 3).  The gradient is pinned against finite
differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np

H = 64


def _shapes(nin, depth):
    out = [("W1", (H, nin)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,))]
    if depth == 3:
        out += [("Wm", (H, H)), ("bm", (H,))]
    return out + [("W3", (4, H)), ("b3", (4,))]


def unpack(p, nin, depth=2):
    p = np.asarray(p, np.float64)
    o = 0
    out = {}
    for name, shape in _shapes(nin, depth):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def n_params(nin, depth=2):
    return sum(int(np.prod(s)) for _, s in _shapes(nin, depth))


def _hidden(w, x, depth):
    """Hidden activations [h1, h2(, h3)] of the inputs x."""
    hs = [np.tanh(x @ w["W1"].T + w["b1"])]
    hs.append(np.tanh(hs[-1] @ w["W2"].T + w["b2"]))
    if depth == 3:
        hs.append(np.tanh(hs[-1] @ w["Wm"].T + w["bm"]))
    return hs


def forward(p, x, nin, depth=2):
    w = unpack(p, nin, depth)
    x = np.asarray(x, np.float64)
    hs = _hidden(w, x, depth)
    o = hs[-1] @ w["W3"].T + w["b3"]
    vn = np.linalg.norm(o[:, :3], axis=1)
    mu = o[:, :3] / vn[:, None]
    kappa = np.logaddexp(0.0, o[:, 3]) + 1e-4
    return mu, kappa, (x, hs, o, vn)


def nll(p, x, y, nin, depth=2):
    """Sum over samples of -log q(y | x) for the vMF law."""
    mu, k, _ = forward(p, x, nin, depth)
    y = np.asarray(y, np.float64)
    log_norm = np.log(k) - np.log(4 * np.pi) - (k + np.log1p(-np.exp(-2 * k)) - np.log(2.0))
    return float(-(log_norm + k * (mu * y).sum(1)).sum())


def grad(p, x, y, nin, depth=2):
    """Gradient of nll by explicit back-propagation (FP64)."""
    w = unpack(p, nin, depth)
    mu, k, (x, hs, o, vn) = forward(p, x, nin, depth)
    y = np.asarray(y, np.float64)
    muy = (mu * y).sum(1)
    dk = 1.0 / np.tanh(k) - 1.0 / k - muy
    dO = np.zeros_like(o)
    dO[:, 3] = dk / (1.0 + np.exp(-o[:, 3]))
    dO[:, :3] = -k[:, None] * (y - mu * muy[:, None]) / vn[:, None]
    g = {"W3": dO.T @ hs[-1], "b3": dO.sum(0)}
    # back through the hidden layers, last to first: the weight that maps layer l-1 to l
    names = ["W1", "W2"] + (["Wm"] if depth == 3 else [])
    bias = {"W1": "b1", "W2": "b2", "Wm": "bm"}
    d = (dO @ w["W3"]) * (1 - hs[-1] ** 2)
    for layer in range(depth - 1, -1, -1):
        name = names[layer]
        inp = x if layer == 0 else hs[layer - 1]
        g[name] = d.T @ inp
        g[bias[name]] = d.sum(0)
        if layer > 0:
            d = (d @ w[name]) * (1 - hs[layer - 1] ** 2)
    return np.concatenate([g[n].ravel() for n, _ in _shapes(nin, depth)])


def init(nin, seed, depth=2):
    """Glorot-uniform weights, zero biases (test parameters drawn on the host)."""
    g = np.random.default_rng(seed)
    parts = []
    for name, shape in _shapes(nin, depth):
        if name.startswith("b"):
            parts.append(np.zeros(shape[0]))
        else:
            fan_out, fan_in = shape
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            parts.append(g.uniform(-lim, lim, size=fan_out * fan_in))
    return np.concatenate(parts)
