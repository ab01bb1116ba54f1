"""Pins of the FP64 learned-proposal oracle: the vMF negative log-likelihood against the
normaliser integrated numerically, and the back-propagated gradient against central
finite differences (independent of the backward formulas)."""
import numpy as np

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


def test_gradient_matches_finite_differences():
    nin = 12
    p = mlp.init(nin, 5) * 2.0
    x = synth.random_unit(4 * 16, 2).reshape(16, 12)
    y = synth.random_unit(16, 3)
    g = mlp.grad(p, x, y, nin)
    rng = np.random.default_rng(0)
    idx = rng.choice(len(p), 60, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (mlp.nll(p + e, x, y, nin) - mlp.nll(p - e, x, y, nin)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
