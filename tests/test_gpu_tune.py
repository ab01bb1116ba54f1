"""The autotuner on the GPU: the tuned launch gives the default launch's sums (the tile
shape changes only the rounding order of the FP32 per-tile sums) and passes the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_07487_gb300 import synth, tune

pytestmark = pytest.mark.gpu

SPACE = {"tile_n": [128, 192, 256], "epi_warps": [4, 8], "raster_m": [8, 16]}


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def test_tuned_plan_matches_default_and_oracle(asd, tmp_path):
    lat = synth.hypercubic(11, 3, True)
    tr = synth.traj_precess(lat.n_sites, 40, seed=3)
    d_tr = torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda()
    tuner = tune.Tuner(path=str(tmp_path / "t.json"))
    best = tuner.tune_plan(asd, lat, 40, 24, 0.5, 20, d_tr, n_t_sample=3, space=SPACE)
    assert set(best) == set(SPACE)
    out = {}
    for name, kw in (("default", {}), ("tuned", best)):
        plan = asd.CorrPlan.for_lattice(lat, 40, 24, 9, 0.5, 20, **kw)
        C = torch.zeros((9, 20), dtype=torch.float64, device="cuda")
        plan.run(d_tr, C)
        assert asd.sync_status() == 0
        out[name] = C.cpu().numpy()
        plan.close()
    np.testing.assert_allclose(out["tuned"], out["default"], rtol=1e-6, atol=1e-6)
    ref = oracle.pair_corr(tr, 24, list(range(9)), oracle.Geometry.of_lattice(lat), 0.5, 20)
    assert oracle.bin_error(out["tuned"], ref).max() <= 1e-5


def test_tuned_batch_matches_oracle(asd):
    probs, trajs, raw = [], [], []
    for k, (L, d) in enumerate(((9, 2), (5, 3), (14, 2))):
        lat = synth.hypercubic(L, d, True)
        w = 1.0 if d == 2 else 0.5
        nb = int(np.floor(np.sqrt(d * (L // 2) ** 2) / w)) + 1
        tr = synth.traj_precess(lat.n_sites, 30, seed=40 + k)
        probs.append((lat, w, nb))
        raw.append(tr)
        trajs.append(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda())
    best = tune.Tuner().tune_batch(asd, probs, 30, 16, trajs, n_t_sample=2, space=SPACE)
    plans = [asd.CorrPlan.for_lattice(lat, 30, 16, 6, w, nb, **best) for lat, w, nb in probs]
    Cs = [torch.zeros((6, nb), dtype=torch.float64, device="cuda") for _, _, nb in probs]
    asd.pair_corr_batched(plans, trajs, Cs)
    assert asd.sync_status() == 0
    for (lat, w, nb), tr, C in zip(probs, raw, Cs):
        ref = oracle.pair_corr(tr, 16, list(range(6)), oracle.Geometry.of_lattice(lat), w, nb)
        assert oracle.bin_error(C.cpu().numpy(), ref).max() <= 1e-5
    for p in plans:
        p.close()
