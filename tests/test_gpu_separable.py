"""GPU parity of the separable phase form (asd_pair_corr_sq_separable) against the FP64
oracle: the pair loop on small cases, the FP64 transform route at full size."""
import numpy as np
import pytest
import torch

import oracle
from oracle import checks
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu

# FP32 transforms within 4096-site slices (about sqrt(4096) * 2^-24 relative to the sum of
# absolute terms), FP64 afterwards: 1e-5 of the largest |Sq| is a wide margin.
TOL = 1e-5


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def sep_gpu(asd, lat, tr, T0, n_t, q, center=False, positions=None, precision="split_bf16"):
    tr4 = np.ascontiguousarray(tr if tr.ndim == 4 else tr[:, None])
    N, S, F, _ = tr4.shape
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, 0.5, 0, precision=precision, S=S,
                                    center=center, q=q, positions=positions)
    Sq = torch.zeros((n_t, len(q)), dtype=torch.float64, device="cuda")
    plan.sq_separable(torch.from_numpy(tr4).cuda(), Sq)
    assert asd.sync_status() == 0
    plan.close()
    return Sq.cpu().numpy()


def rel(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("center", [False, True])
def test_positions_vs_pair_oracle(asd, center):
    """Jittered open cube, 13 q (a partial chunk), 2 samples, every displacement."""
    lat = synth.hypercubic(7, 3, False, jitter=0.1, seed=3)
    q = synth.q_vectors_glass()[::5]
    tr = synth.traj_precess(lat.n_sites, 30, seed=8, S=2)
    got = sep_gpu(asd, lat, tr, 20, 11, q, center=center)
    ref = oracle.pair_corr(tr, 20, list(range(11)), oracle.Geometry.of_lattice(lat), 0.5, 1,
                           q=q, center=center)
    assert rel(got, ref["Sq_sum"]) <= TOL


def test_lattice_q_path_vs_pair_oracle(asd):
    """Periodic square lattice with the high-symmetry q path (integer coordinates); more
    than one 4096-site slice, so the FP64 slice sums are exercised."""
    lat = synth.hypercubic(72, 2, True)
    q = synth.q_path_square(72)[::7]
    tr = synth.traj_precess(lat.n_sites, 16, seed=2)
    got = sep_gpu(asd, lat, tr, 10, 6, q)
    ref = checks.separable_phase_sum(tr, 10, list(range(6)), lat.coords.astype(np.float64), q)
    assert rel(got, ref) <= TOL
    # and the pair loop on a smaller lattice of the same kind
    lat2 = synth.hypercubic(12, 2, True)
    q2 = synth.q_path_square(12)
    tr2 = synth.traj_precess(lat2.n_sites, 16, seed=4)
    got2 = sep_gpu(asd, lat2, tr2, 10, 6, q2)
    ref2 = oracle.pair_corr(tr2, 10, list(range(6)), oracle.Geometry.of_lattice(lat2), 1.0, 1, q=q2)
    assert rel(got2, ref2["Sq_sum"]) <= TOL


def test_matches_fused_phase_epilogue(asd):
    """The two GPU evaluations of the same sum (fused pair kernel and separable route)
    agree to the accuracy of the FP32-accurate fused form."""
    lat = synth.hypercubic(10, 3, False, jitter=0.1, seed=5)
    q = synth.q_vectors_glass()[::4]
    tr = synth.traj_precess(lat.n_sites, 40, seed=9)
    sep = sep_gpu(asd, lat, tr, 24, 9, q)
    plan = asd.CorrPlan.for_lattice(lat, 40, 24, 9, 0.5, 0, precision="split_bf16", q=q)
    Sq = torch.zeros((9, len(q)), dtype=torch.float64, device="cuda")
    plan.run(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda(), None, Sq)
    assert asd.sync_status() == 0
    plan.close()
    ref = oracle.pair_corr(tr, 24, list(range(9)), oracle.Geometry.of_lattice(lat), 0.5, 1, q=q)
    assert rel(sep, ref["Sq_sum"]) <= TOL
    # the fused split-BF16 sums at the accuracy bar, per (t, q) in units of that q's
    # magnitude sum
    assert oracle.phase_error(Sq.cpu().numpy(), ref).max() <= 1e-5


@pytest.mark.slow
def test_glass_full_size_vs_fp64_transform(asd):
    """64^3 jittered glass (262144 sites, F = 640, T0 = 512, 64 q), all 128 displacements
    on the GPU, checked at 3 of them against the FP64 transform route."""
    cfg = synth.cfg_glass64()
    lat = cfg.lattice
    tr = synth.traj_precess(lat.n_sites, cfg.F, seed=23083)
    got = sep_gpu(asd, lat, tr, cfg.T0, cfg.n_t, cfg.q)
    t_sel = [0, 63, 127]
    ref = checks.separable_phase_sum(tr, cfg.T0, t_sel, lat.pos, cfg.q)
    assert rel(got[t_sel], ref) <= TOL
