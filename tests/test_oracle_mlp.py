"""Pins of the FP64 learned-proposal oracle: the vMF negative log-likelihood against the
normaliser integrated numerically, and the back-propagated gradient against central
finite differences (independent of the backward formulas)."""
import numpy as np
import pytest

from oracle import mlp
from paper_2308_07487_gb300 import synth


def test_vmf_density_integrates_to_one():
    """exp(-NLL) integrated over the sphere is 1 for any (mu, kappa) the network emits."""
    nin = 12
    p = mlp.init(nin, 3)
    x = synth.random_unit(4 * 5, 1).reshape(5, 12)
    mu, k, _ = mlp.forward(p, x, nin)
    # integrate over the sphere in coordinates about mu: density depends on cos only
    c = np.linspace(-1, 1, 200001)
    for kk in k:
        dens = kk / (4 * np.pi * np.sinh(kk)) * np.exp(kk * c)
        total = 2 * np.pi * np.trapezoid(dens, c)
        assert abs(total - 1.0) < 1e-8
    # NLL of y = mu is -log of the peak density
    y = mu
    ref = -np.log(k / (4 * np.pi * np.sinh(k)) * np.exp(k)).sum()
    assert abs(mlp.nll(p, x, y, nin) - ref) < 1e-9 * abs(ref)


@pytest.mark.parametrize("depth", [2, 3])
def test_gradient_matches_finite_differences(depth):
    nin = 12
    p = mlp.init(nin, 5, depth) * 2.0
    assert len(p) == mlp.n_params(nin, depth)
    x = synth.random_unit(4 * 16, 2).reshape(16, 12)
    y = synth.random_unit(16, 3)
    g = mlp.grad(p, x, y, nin, depth)
    rng = np.random.default_rng(0)
    # every layer's weights and biases are sampled (the blocks of the packed vector)
    idx = rng.choice(len(p), 80, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (mlp.nll(p + e, x, y, nin, depth) - mlp.nll(p - e, x, y, nin, depth)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_three_layers_reduce_to_two_with_an_identity_like_layer():
    """A third hidden layer that passes its input through (Wm = a * identity, bm = 0 with a
    small a and the output weights scaled by 1/a) reproduces the two-layer network to
    first order in a: a check of the packed layout and of the extra layer's place."""
    nin, a = 12, 1e-4
    p2 = mlp.init(nin, 7)
    w2 = mlp.unpack(p2, nin)
    parts = [w2["W1"].ravel(), w2["b1"], w2["W2"].ravel(), w2["b2"],
             (a * np.eye(mlp.H)).ravel(), np.zeros(mlp.H), (w2["W3"] / a).ravel(), w2["b3"]]
    p3 = np.concatenate(parts)
    x = synth.random_unit(4 * 8, 4).reshape(8, 12)
    mu2, k2, _ = mlp.forward(p2, x, nin)
    mu3, k3, _ = mlp.forward(p3, x, nin, 3)
    np.testing.assert_allclose(mu3, mu2, atol=1e-6)
    np.testing.assert_allclose(k3, k2, rtol=1e-6)
