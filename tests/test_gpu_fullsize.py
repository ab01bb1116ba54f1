"""Parity at the full workload sizes, in the launch configuration bench.py times.

* 40^3 periodic lattice, N = 64000, F = 1200, T0 = 1000, 200 displacements, 70 bins:
  the whole split-BF16 launch against the FFT cross-correlation route (exact FP64, an
  independent algorithm), every bin of a spread of displacements, in C(b,t) units
  (|C| <= 1, C(0,0) = 1): |C_gpu - C_ref| <= 1e-5; plus rows 0..4 against the loop
  oracle with the per-bin metric.
* 64^3 jittered +-J glass (262144 sites, open, 256 bins, 64 q): 32 random 16-row blocks
  of the bins and of the phase sums against the loop oracle at 4 displacements.
* 96-sample uneven ensemble (N_s up to 40000, F = 320, T0 = 256, 64 displacements), one
  batched split-BF16 launch as the bench runs it: every problem against the FFT route.
* 128^2 lattice with 64 starts concatenated along K (K = 98304, F = 576, T0 = 512,
  64 displacements): rows against the loop oracle, C(0,0) = 1 on the full launch.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import checks
from paper_2308_07487_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def test_cubic40_full_launch_vs_fft(asd):
    cfg = synth.cfg_cubic40()
    lat = cfg.lattice
    tr = synth.traj_precess(lat.n_sites, cfg.F, seed=23082)
    d_tr = torch.from_numpy(tr).cuda()
    plan = asd.CorrPlan.for_lattice(lat, cfg.F, cfg.T0, cfg.n_t, cfg.w, cfg.n_bins,
                                    precision="split_bf16")
    C = torch.zeros((cfg.n_t, cfg.n_bins), dtype=torch.float64, device="cuda")
    plan.run(d_tr, C)
    assert asd.sync_status() == 0
    got = C.cpu().numpy()
    counts = plan.counts()
    t_list = [0, 1, 7, 50, 123, 199]
    ref = checks.lattice_fft_corr(tr, cfg.T0, t_list, lat.coords, lat.L, True, cfg.w, cfg.n_bins)
    n = counts.astype(np.float64)
    occ = n > 0                       # no lattice distance falls in [0.5, 1): bin 1 is empty
    err = np.abs(got[t_list][:, occ] - ref[:, occ]) / (cfg.T0 * n[occ])
    assert err.max() <= 1e-5, err.max()
    assert np.abs(got[t_list][:, ~occ]).max(initial=0.0) == 0.0
    assert np.abs(ref[:, ~occ]).max(initial=0.0) < 1e-6 * cfg.T0
    # the loop oracle on 4 rows x all columns, per-bin metric
    rows = (0, 4)
    Cr = torch.zeros_like(C)
    plan.run(d_tr, Cr, rows=rows)
    r = oracle.pair_corr(tr, cfg.T0, [0, 199], oracle.Geometry.of_lattice(lat), cfg.w,
                         cfg.n_bins, rows=rows)
    assert oracle.bin_error(Cr.cpu().numpy()[[0, 199]], r).max() <= 1e-5
    plan.close()


def test_glass_rows_bins_and_phase(asd):
    """32 seeded random blocks of 16 rows (each against all 262144 columns) at 4
    displacements spread over [0, 127]: every (t, q) of the phase sums within 1e-5 of the
    loop oracle in units of the q's magnitude sum; every bin holding at least 16 pairs of
    the block within 1e-5 in units of its magnitude sum, and every bin (the far bins of a
    16-row block hold single pairs) within 1e-5 of the sum of |products| (the rounding
    scale: plain FP32 lands at 5e-6 of it, 7e-6 of |G| on single pairs)."""
    cfg = synth.cfg_glass64()
    lat = cfg.lattice
    tr = synth.traj_precess(lat.n_sites, cfg.F, seed=23083)
    d_tr = torch.from_numpy(tr).cuda()
    plan = asd.CorrPlan.for_lattice(lat, cfg.F, cfg.T0, cfg.n_t, cfg.w, cfg.n_bins,
                                    precision="split_bf16", q=cfg.q)
    t_sel = [0, 42, 85, 127]
    starts = np.sort(np.random.default_rng(23083).choice(lat.n_sites // 16, 32, replace=False)) * 16
    geo = oracle.Geometry.of_lattice(lat)
    worst_b, worst_q, worst_p = 0.0, 0.0, 0.0
    for i0 in starts:
        rows = (int(i0), int(i0) + 16)
        C = torch.zeros((cfg.n_t, cfg.n_bins), dtype=torch.float64, device="cuda")
        Sq = torch.zeros((cfg.n_t, len(cfg.q)), dtype=torch.float64, device="cuda")
        plan.run(d_tr, C, Sq, rows=rows)
        assert asd.sync_status() == 0
        r = oracle.pair_corr(tr, cfg.T0, t_sel, geo, cfg.w, cfg.n_bins, q=cfg.q, rows=rows)
        c = C.cpu().numpy()[t_sel]
        worst_b = max(worst_b, float(oracle.sampled_bin_error(c, r).max()))
        worst_p = max(worst_p, float(oracle.rounding_ratio(c, r).max()))
        worst_q = max(worst_q, float(oracle.phase_error(Sq.cpu().numpy()[t_sel], r).max()))
    plan.close()
    assert worst_b <= 1e-5, worst_b
    assert worst_p <= 1e-5, worst_p
    assert worst_q <= 1e-5, worst_q


def test_ensemble96_batched_vs_fft(asd):
    F, T0, n_t = 320, 256, 64
    t_list = [0, 1, 31, 63]
    probs = []
    for k, (d, L) in enumerate(synth.ensemble_sizes(96)):
        lat = synth.hypercubic(L, d, True, J=1.0)
        w = 1.0 if d == 2 else 0.5
        nb = int((d * (L // 2) ** 2) ** 0.5 / w) + 1
        tr = synth.traj_precess(lat.n_sites, F, seed=23084 + k)
        plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision="split_bf16",
                                        tile_n=256)
        probs.append((lat, w, nb, tr, plan, torch.from_numpy(tr[:, None].copy()).cuda(),
                      torch.zeros((n_t, nb), dtype=torch.float64, device="cuda")))
    asd.pair_corr_batched([p[4] for p in probs], [p[5] for p in probs], [p[6] for p in probs])
    assert asd.sync_status() == 0
    worst = 0.0
    for lat, w, nb, tr, plan, _, C in probs:
        n = plan.counts().astype(np.float64)
        ref = checks.lattice_fft_corr(tr, T0, t_list, lat.coords, lat.L, True, w, nb)
        got = C.cpu().numpy()[t_list]
        occ = n > 0
        worst = max(worst, float((np.abs(got[:, occ] - ref[:, occ]) / (T0 * n[occ])).max()))
        assert np.abs(got[:, ~occ]).max(initial=0.0) == 0.0
        plan.close()
    assert worst <= 1e-5, worst


def test_learned_config_k98304(asd):
    L, S, F, T0, n_t = 128, 64, 576, 512, 64
    lat = synth.hypercubic(L, 2, True, J=1.0)
    # [N][S][F][3], generated one start at a time (bounded host memory)
    tr = np.empty((lat.n_sites, S, F, 3), np.float32)
    for s in range(S):
        tr[:, s] = synth.traj_precess(lat.n_sites, F, seed=23085 + s)[:, 0]
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, 1.0, 91, precision="split_bf16", S=S)
    d_tr = torch.from_numpy(tr).cuda()
    C = torch.zeros((n_t, 91), dtype=torch.float64, device="cuda")
    plan.run(d_tr, C)
    Cr = torch.zeros_like(C)
    rows = (5000, 5004)
    plan.run(d_tr, Cr, rows=rows)
    assert asd.sync_status() == 0
    r = oracle.pair_corr(tr, T0, [0, 63], oracle.Geometry.of_lattice(lat), 1.0, 91, rows=rows)
    assert oracle.bin_error(Cr.cpu().numpy()[[0, 63]], r).max() <= 1e-5
    # the full launch at any size: C(0, 0) = 1 for unit spins (self pairs only in bin 0)
    n = plan.counts().astype(np.float64)
    c00 = C.cpu().numpy()[0, 0] / (S * T0 * n[0])
    assert abs(c00 - 1.0) <= 1e-5, c00
    plan.close()
