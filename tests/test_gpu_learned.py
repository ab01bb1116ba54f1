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


def _weight_ranges(nin, depth):
    """[start, end) of every weight matrix in the packed parameter vector."""
    out, o = [], 0
    for name, shape in omlp._shapes(nin, depth):
        n = int(np.prod(shape))
        if not name.startswith("b"):
            out.append((o, o + n))
        o += n
    return out


def _bf16_point(p, nin, depth=2):
    """The oracle evaluates at the weights the GPU uses: BF16-rounded W, FP32 biases."""
    t = torch.from_numpy(p.astype(np.float32))
    q = t.clone()
    for a, b in _weight_ranges(nin, depth):
        q[a:b] = t[a:b].to(torch.bfloat16).float()
    return q.double().numpy()


@pytest.mark.parametrize("depth", [2, 3])
def test_loss_and_gradient_match_oracle(asd, depth):
    nin = 12
    p = omlp.init(nin, 7, depth) * 1.5
    net = asd.Mlp(nin, p, depth=depth)
    x = synth.random_unit(4 * 3000, 1).reshape(3000, 12)
    y = synth.random_unit(3000, 2)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net.loss_grad(dx, dy)
    assert asd.sync_status() == 0
    pb = _bf16_point(p, nin, depth)
    ref_l = omlp.nll(pb, x, y, nin, depth)
    ref_g = omlp.grad(pb, x, y, nin, depth)
    assert abs(net.loss.item() - ref_l) <= 1e-5 * abs(ref_l)
    g = net.grad.cpu().double().numpy()
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)
    assert np.abs(g - ref_g).max() <= 1e-3 * np.abs(ref_g).max()


@pytest.mark.parametrize("depth", [2, 3])
def test_library_initialiser(asd, depth):
    """asd_mlp_init: Glorot-uniform weights inside +-sqrt(6 / (fan_in + fan_out)) with the
    moments of that uniform law, zero biases, the BF16 copy equal to the round-to-nearest
    of the parameters, the same draw for the same seed and a different one otherwise."""
    nin, H = 12, 64
    a = asd.Mlp(nin, seed=7, depth=depth)
    b = asd.Mlp(nin, seed=7, depth=depth)
    c = asd.Mlp(nin, seed=8, depth=depth)
    assert asd.sync_status() == 0
    p = a.params.cpu().double().numpy()
    assert p.shape == (omlp.n_params(nin, depth),)
    assert np.array_equal(p, b.params.cpu().double().numpy())
    assert not np.array_equal(p, c.params.cpu().double().numpy())
    w = omlp.unpack(p, nin, depth)
    layers = (("W1", nin + H), ("W2", 2 * H)) + ((("Wm", 2 * H),) if depth == 3 else ()) + \
        (("W3", H + 4),)
    for name, fan in layers:
        lim = math.sqrt(6.0 / fan)
        x = w[name].ravel()
        assert np.abs(x).max() <= lim and np.abs(x).max() > 0.9 * lim, name
        # mean 0 and variance lim^2 / 3 of U(-lim, lim), within 5 standard errors
        n = x.size
        assert abs(x.mean()) <= 5 * lim / math.sqrt(3 * n), name
        assert abs(x.var() / (lim * lim / 3) - 1) <= 5 * math.sqrt(0.8 / n), name
    for name in ("b1", "b2", "b3") + (("bm",) if depth == 3 else ()):
        assert not w[name].any(), name
    idx = np.concatenate([np.arange(a0, b0) for a0, b0 in _weight_ranges(nin, depth)])
    assert np.array_equal(a.wb.float().cpu().double().numpy(), _bf16_point(p, nin, depth)[idx])


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


def _train(asd, sysm, lat, T, S, seed, sweeps0=300, snaps=40, steps=600, B=8192, depth=2):
    """Train a fresh network (library initialiser) on plain Metropolis configurations."""
    n_in = 3 * lat.nbr.shape[1]
    sp = torch.from_numpy(synth.random_unit(S * lat.n_sites, seed).reshape(S, lat.n_sites, 3)).cuda()
    sysm.thermalize(sp, T, sweeps0, asd.ASD_METROPOLIS, cone=0.0, adapt=True, seed=seed)
    xs, ys = [], []
    for k in range(snaps):
        sysm.thermalize(sp, T, 4, asd.ASD_METROPOLIS, cone=0.0, adapt=True, seed=seed,
                        counter=sweeps0 + 4 * k)
        x = torch.empty((S * lat.n_sites, n_in), device="cuda")
        y = torch.empty((S * lat.n_sites, 3), device="cuda")
        sysm.gather(sp, x, y)
        xs.append(x)
        ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys)
    n = X.shape[0]
    net = asd.Mlp(n_in, seed=seed + 10, depth=depth)
    g = torch.Generator(device="cuda").manual_seed(0)
    for it in range(steps):
        idx = torch.randint(0, n, (B,), device="cuda", generator=g)
        net.grad.zero_()
        net.loss.zero_()
        net.loss_grad(X[idx].contiguous(), Y[idx].contiguous())
        net.adam(lr=3e-3 if it < 2 * steps // 3 else 1e-3, scale=1.0 / B)
    return net, sp, X, Y


@pytest.fixture(scope="module")
def square16(asd):
    """16^2 periodic AFM (J = +1) at T = 0.7 with a network trained on 40 x 64 Metropolis
    configurations."""
    L, T, S = 16, 0.7, 64
    lat = synth.hypercubic(L, 2, True, J=1.0)
    sysm = asd.System(lat)
    net, sp, X, Y = _train(asd, sysm, lat, T, S, seed=1)
    assert asd.sync_status() == 0
    return dict(lat=lat, sysm=sysm, net=net, sp=sp, X=X, Y=Y, T=T, S=S)


def test_training_reaches_heatbath(asd, square16):
    """Trained from the library initialiser, the network's NLL comes within 0.03 nats per
    site of the exact heat-bath conditional's (the best any proposal can do)."""
    net, X, Y, T = square16["net"], square16["X"], square16["Y"], square16["T"]
    net.grad.zero_()
    net.loss.zero_()
    net.loss_grad(X[:65536].contiguous(), Y[:65536].contiguous())
    assert asd.sync_status() == 0
    trained = net.loss.item() / 65536
    opt = _heatbath_nll(X[:65536].double().cpu().numpy(), Y[:65536].double().cpu().numpy(), 1 / T) / 65536
    uniform = math.log(4 * math.pi)
    assert trained < opt + 0.03, (trained, opt, uniform)


def _tau_int(E):
    """Integrated autocorrelation time of per-chain series E [chains][measurements]: the
    chain-averaged normalised autocorrelation summed to its first non-positive lag."""
    X = E - E.mean(axis=1, keepdims=True)
    var = (X * X).mean()
    n = X.shape[1]
    tau = 0.5
    for k in range(1, n // 3):
        r = float((X[:, :n - k] * X[:, k:]).mean() / var)
        if r <= 0:
            break
        tau += r
    return tau


def test_learned_proposal_decorrelates_faster(asd, square16):
    """What the trained network gains: higher acceptance than plain Metropolis with a
    uniform trial spin and a shorter integrated autocorrelation time of the energy (one
    sweep between measurements, 64 chains x 120 measurements, fixed seeds)."""
    lat, sysm, net, sp, T = (square16[k] for k in ("lat", "sysm", "net", "sp", "T"))
    nbr = torch.from_numpy(lat.nbr).long().cuda()
    res = {}
    for name, prop, kw in (("learned", asd.ASD_LEARNED, {"net": net}),
                           ("metropolis", asd.ASD_METROPOLIS, {"cone": 0.0})):
        s2 = sp.clone()
        sysm.thermalize(s2, T, 100, prop, seed=3, **kw)
        es, ac, pr = [], 0, 0
        for k in range(120):
            st = sysm.thermalize(s2, T, 1, prop, seed=3, counter=100 + k, stats=True, **kw)
            pr += st[0]
            ac += st[1]
            y = s2.double()
            e = sum((y * y[:, nbr[:, a]]).sum(dim=(1, 2)) for a in range(nbr.shape[1]))
            es.append((e / 2 / lat.n_sites).cpu().numpy())
        res[name] = (ac / pr, _tau_int(np.stack(es, 1)))
    assert asd.sync_status() == 0
    (acc_l, tau_l), (acc_m, tau_m) = res["learned"], res["metropolis"]
    assert acc_l > 0.7 and acc_l > acc_m + 0.2, res
    assert tau_l < 0.6 * tau_m, res


@pytest.mark.parametrize("depth", [2, 3])
def test_learned_chain_is_exact_open_chain(asd, depth):
    """Exactness of the Metropolis-Hastings correction: on an open chain the bond angles
    are independent and <S_i . S_i+1> = -L(beta J) (Langevin function) exactly.  A network
    (two or three hidden layers) trained on the chain (2 neighbours, 6 inputs) drives the
    learned proposal; the bond average over 4095 bonds x 16 chains x 60 snapshots must
    agree with the closed form within 5 standard errors of 12 block means (about 8e-4)."""
    n, S, T = 4096, 16, 0.5
    lat = synth.open_chain(n, J=1.0)
    sysm = asd.System(lat)
    net, sp, _, _ = _train(asd, sysm, lat, T, S, seed=21, sweeps0=200, snaps=16, steps=300,
                           depth=depth)
    s2 = sp.clone()
    sysm.thermalize(s2, T, 50, asd.ASD_LEARNED, net=net, seed=5)
    snaps, ac, pr = [], 0, 0
    for k in range(60):
        st = sysm.thermalize(s2, T, 2, asd.ASD_LEARNED, net=net, seed=5, counter=50 + 2 * k,
                             stats=True)
        pr += st[0]
        ac += st[1]
        y = s2.double()
        snaps.append((y[:, :-1] * y[:, 1:]).sum(-1).mean().item())
    assert asd.sync_status() == 0
    blocks = np.array(snaps).reshape(12, 5).mean(1)
    sem = blocks.std(ddof=1) / math.sqrt(len(blocks))
    bJ = 1.0 / T
    ref = -(1 / math.tanh(bJ) - 1 / bJ)
    assert ac / pr > 0.5, ac / pr
    assert abs(np.mean(snaps) - ref) < 5 * sem, (np.mean(snaps), ref, sem)
