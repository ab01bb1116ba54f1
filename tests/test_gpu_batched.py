"""Batched uneven ensemble (one persistent launch over many problems) and CUDA-graph
capture of it, against the FP64 oracle and against per-problem launches."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def _ensemble(n=6, F=30, T0=16, n_t=10, seed=5, drop=False):
    g = np.random.default_rng(seed)
    out = []
    for k in range(n):
        d = 2 + (k % 2)
        L = int(g.integers(5, 14 if d == 2 else 7))
        w = 1.0 if d == 2 else 0.5
        lat = synth.hypercubic(L, d, True)
        rmax2 = d * (L // 2) ** 2
        n_bins = int(np.floor(np.sqrt(rmax2) / w)) + 1
        if drop and k % 2 == 0:
            n_bins = max(2, n_bins // 2)   # the far pairs of this problem are dropped
        tr = synth.traj_precess(lat.n_sites, F, seed=100 + k)
        out.append((lat, tr, w, n_bins))
    return out, F, T0, n_t


@pytest.mark.parametrize("form,drop", [("split_bf16", False), ("bf16", False),
                                       ("split_bf16", True)])
def test_batched_matches_oracle_and_single_launches(asd, form, drop):
    ens, F, T0, n_t = _ensemble(drop=drop)
    plans, trajs, Cs, Cs1 = [], [], [], []
    for lat, tr, w, nb in ens:
        p = asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision=form, tile_n=128)
        plans.append(p)
        trajs.append(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda())
        Cs.append(torch.zeros((n_t, nb), dtype=torch.float64, device="cuda"))
        Cs1.append(torch.zeros((n_t, nb), dtype=torch.float64, device="cuda"))
    asd.pair_corr_batched(plans, trajs, Cs)
    for p, t, c in zip(plans, trajs, Cs1):
        p.run(t, c)
    assert asd.sync_status() == 0
    tol = 1e-5 if form == "split_bf16" else 4 * 2.0 ** -8
    for (lat, tr, w, nb), c, c1 in zip(ens, Cs, Cs1):
        ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb)
        assert oracle.bin_error(c.cpu().numpy(), ref).max() <= tol
        # same arithmetic, only the tile order differs: FP64 reduction order only
        np.testing.assert_allclose(c.cpu().numpy(), c1.cpu().numpy(), rtol=1e-9, atol=1e-9)
    for p in plans:
        p.close()


def test_batched_graph_capture_replay(asd):
    ens, F, T0, n_t = _ensemble(n=4, seed=9)
    plans, trajs, Cs = [], [], []
    for lat, tr, w, nb in ens:
        plans.append(asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision="split_bf16",
                                              tile_n=128))
        trajs.append(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda())
        Cs.append(torch.zeros((n_t, nb), dtype=torch.float64, device="cuda"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        asd.pair_corr_batched(plans, trajs, Cs, stream=s)   # uploads the work list
    torch.cuda.synchronize()
    first = [c.clone() for c in Cs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for c in Cs:
            c.zero_()
        asd.pair_corr_batched(plans, trajs, Cs, stream=s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert asd.sync_status() == 0
    for a, b in zip(first, Cs):
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-9, atol=1e-9)
    for p in plans:
        p.close()


def test_graph_survives_a_batch_led_by_another_plan(asd):
    """The work list of a batched launch lives in its first plan: a larger batch led by
    another plan, run between capture and replay, leaves the captured graph's work list
    alone, and both batches match the oracle."""
    ens_a, F, T0, n_t = _ensemble(n=3, seed=11)
    ens_b, _, _, _ = _ensemble(n=7, seed=12)

    def make(ens):
        plans, trajs, Cs = [], [], []
        for lat, tr, w, nb in ens:
            plans.append(asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb,
                                                  precision="split_bf16", tile_n=128))
            trajs.append(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda())
            Cs.append(torch.zeros((n_t, nb), dtype=torch.float64, device="cuda"))
        return plans, trajs, Cs

    pa, ta, ca = make(ens_a)
    pb, tb, cb = make(ens_b)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        asd.pair_corr_batched(pa, ta, ca, stream=s)   # uploads batch A's work list
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for c in ca:
            c.zero_()
        asd.pair_corr_batched(pa, ta, ca, stream=s)
    with torch.cuda.stream(s):
        asd.pair_corr_batched(pb, tb, cb, stream=s)   # uploads batch B's work list
    g.replay()
    torch.cuda.synchronize()
    assert asd.sync_status() == 0
    for (lat, tr, w, nb), c in zip(ens_a + ens_b, ca + cb):
        ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb)
        assert oracle.bin_error(c.cpu().numpy(), ref).max() <= 1e-5
    for p in pa + pb:
        p.close()
