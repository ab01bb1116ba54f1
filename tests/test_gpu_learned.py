"""Learned vMF proposal: GPU loss/gradient against the FP64 oracle, training on plain
Metropolis configurations, and Metropolis-Hastings sampling with the trained network
compared with the exact heat-bath chain (energy) and with plain Metropolis (acceptance,
decorrelation)."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def _bf16_point(p, nin):
    """The oracle evaluates at the weights the GPU uses: BF16-rounded W, FP32 biases."""
    t = torch.from_numpy(p.astype(np.float32))
    q = t.clone()
    H = 64
    for a, b in ((0, H * nin), (H * nin + H, H * nin + H + H * H),
                 (H * nin + 2 * H + H * H, H * nin + 2 * H + H * H + 4 * H)):
        q[a:b] = t[a:b].to(torch.bfloat16).float()
    return q.double().numpy()


def test_loss_and_gradient_match_oracle(asd):
    nin = 12
    p = omlp.init(nin, 7) * 1.5
    net = asd.Mlp(nin, p)
    x = synth.random_unit(4 * 3000, 1).reshape(3000, 12)
    y = synth.random_unit(3000, 2)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net.loss_grad(dx, dy)
    assert asd.sync_status() == 0
    pb = _bf16_point(p, nin)
    ref_l = omlp.nll(pb, x, y, nin)
    ref_g = omlp.grad(pb, x, y, nin)
    assert abs(net.loss.item() - ref_l) <= 1e-5 * abs(ref_l)
    g = net.grad.cpu().double().numpy()
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)
    assert np.abs(g - ref_g).max() <= 1e-3 * np.abs(ref_g).max()


def _heatbath_nll(x, y, beta, J=1.0):
    """NLL of the exact conditional vMF(-h/|h|, beta|h|) with h = J * (sum of neighbours)."""
    h = J * x.reshape(len(x), -1, 3).sum(1)
    hn = np.linalg.norm(h, axis=1)
    k = np.maximum(beta * hn, 1e-12)
    mu = -h / np.maximum(hn, 1e-12)[:, None]
    return float(-(np.log(k) - np.log(4 * np.pi) - (k + np.log1p(-np.exp(-2 * k)) - np.log(2.0))
                   + k * (mu * y).sum(1)).sum())


def _energy_per_site(y, lat):
    e = 0.0
    for k in range(lat.nbr.shape[1]):
        e += (lat.J[:, k][None, :, None] * y * y[:, lat.nbr[:, k]]).sum()
    return e / 2 / (y.shape[0] * lat.n_sites)


def test_training_reaches_heatbath_and_learned_chain_is_exact(asd):
    L, T, S = 16, 0.7, 64
    lat = synth.hypercubic(L, 2, True, J=1.0)
    sysm = asd.System(lat)
    sp = torch.from_numpy(synth.random_unit(S * lat.n_sites, 5).reshape(S, lat.n_sites, 3)).cuda()
    sysm.thermalize(sp, T, 300, asd.ASD_METROPOLIS, cone=0.0, adapt=True, seed=1)
    xs, ys = [], []
    for k in range(40):
        sysm.thermalize(sp, T, 4, asd.ASD_METROPOLIS, cone=0.0, adapt=True, seed=1,
                        counter=300 + 4 * k)
        x = torch.empty((S * lat.n_sites, 12), device="cuda")
        y = torch.empty((S * lat.n_sites, 3), device="cuda")
        sysm.gather(sp, x, y)
        xs.append(x)
        ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys)
    n = X.shape[0]
    net = asd.Mlp(12, omlp.init(12, 11))
    g = torch.Generator(device="cuda").manual_seed(0)
    B = 8192
    for it in range(600):
        idx = torch.randint(0, n, (B,), device="cuda", generator=g)
        net.grad.zero_()
        net.loss.zero_()
        net.loss_grad(X[idx].contiguous(), Y[idx].contiguous())
        net.adam(lr=3e-3 if it < 400 else 1e-3, scale=1.0 / B)
    net.grad.zero_()
    net.loss.zero_()
    net.loss_grad(X[:65536].contiguous(), Y[:65536].contiguous())
    assert asd.sync_status() == 0
    trained = net.loss.item() / 65536
    opt = _heatbath_nll(X[:65536].double().cpu().numpy(), Y[:65536].double().cpu().numpy(), 1 / T) / 65536
    uniform = math.log(4 * math.pi)
    assert trained < opt + 0.03, (trained, opt, uniform)

    # learned-proposal MH chain vs heat-bath chain: same energy; higher acceptance than
    # plain Metropolis with a uniform trial spin
    e = {}
    acc = {}
    for name, prop, kw in (("learned", asd.ASD_LEARNED, {"net": net}),
                           ("heatbath", asd.ASD_HEATBATH, {}),
                           ("metropolis", asd.ASD_METROPOLIS, {"cone": 0.0})):
        s2 = sp.clone()
        sysm.thermalize(s2, T, 100, prop, seed=3, **kw)
        es, ac, pr = [], 0, 0
        for k in range(30):
            st = sysm.thermalize(s2, T, 5, prop, seed=3, counter=100 + 5 * k, stats=True, **kw)
            pr += st[0]
            ac += st[1]
            es.append(_energy_per_site(s2.double().cpu().numpy(), lat))
        e[name] = (np.mean(es), np.std(es) / math.sqrt(len(es)))
        acc[name] = ac / pr
    assert acc["learned"] > 0.7 and acc["learned"] > acc["metropolis"] + 0.2, acc
    d = abs(e["learned"][0] - e["heatbath"][0])
    assert d < 4 * math.hypot(e["learned"][1], e["heatbath"][1]) + 2e-3, e
