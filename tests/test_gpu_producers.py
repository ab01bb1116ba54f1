"""GPU parity of the trajectory producers (asd_ll_integrate, asd_thermalize) against the
FP64 oracle, plus closed-form statistics of the in-kernel Philox sampling."""
import math

import numpy as np
import pytest
import torch

from oracle import dynamics as dyn
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def test_ll_matches_fp64_rk4(asd):
    """FP32 RK4 vs FP64 RK4 over 40 frames (stride 2, dt = 0.01): differences stay at
    FP32 rounding level (atol 2e-5 after 80 steps)."""
    lat = synth.hypercubic(10, 2, True, J=-1.0, Hz=0.5)
    S, F, stride = 2, 41, 2
    s0 = synth.random_unit(S * lat.n_sites, 12).reshape(S, lat.n_sites, 3)
    ref = dyn.ll_rk4(s0.astype(np.float64), lat.nbr, lat.J, lat.Hz, 0.01, F, stride)
    sysm = asd.System(lat)
    d0 = torch.from_numpy(s0).cuda()
    traj = torch.zeros((lat.n_sites, S, F, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(d0)
    sysm.ll_integrate(d0, 0.01, F, stride, traj, out)
    assert asd.sync_status() == 0
    got = traj.cpu().numpy()
    assert np.abs(got - ref).max() < 2e-5
    np.testing.assert_allclose(out.cpu().numpy(), np.transpose(got[:, :, -1], (1, 0, 2)), atol=0)


def test_ll_conserves_total_spin(asd):
    lat = synth.hypercubic(12, 3, True, J=1.0)
    s0 = torch.from_numpy(synth.random_unit(lat.n_sites, 4)[None]).cuda()
    F = 101
    traj = torch.zeros((lat.n_sites, 1, F, 3), dtype=torch.float32, device="cuda")
    asd.System(lat).ll_integrate(s0, 0.01, F, 1, traj)
    M = traj.double().sum(0)[0]
    assert (M - M[:1]).abs().max().item() < 1e-3   # FP32 sums of 1728 spins


@pytest.mark.parametrize("proposal,cone", [("metropolis", 0.0), ("metropolis", 0.6),
                                           ("heatbath", 0.0)])
def test_mc_sweeps_match_oracle_given_uniforms(asd, proposal, cone):
    lat = synth.hypercubic(12, 2, True, J=1.0, Hz=0.3)
    S, sweeps, T = 2, 3, 0.8
    g = np.random.default_rng(5)
    u = g.random((sweeps, S, lat.n_sites, 4)).astype(np.float32)
    u[..., :2] = 1.0 - u[..., :2]
    s0 = synth.random_unit(S * lat.n_sites, 9).reshape(S, lat.n_sites, 3)
    Y = s0.astype(np.float64)
    for k in range(sweeps):
        Y, _, _ = dyn.mc_sweep(Y, lat.nbr, lat.J, lat.Hz, T, u[k].astype(np.float64), lat.colors,
                               proposal, cone=cone)
    sp = torch.from_numpy(s0.copy()).cuda()
    pid = asd.ASD_HEATBATH if proposal == "heatbath" else asd.ASD_METROPOLIS
    asd.System(lat).thermalize(sp, T, sweeps, pid, cone=cone, uniforms=torch.from_numpy(u).cuda())
    assert asd.sync_status() == 0
    d = np.abs(sp.cpu().numpy() - Y).max(-1)
    # identical accept decisions: every site within FP32 rounding of the FP64 sweep
    assert (d > 1e-4).mean() == 0.0, f"{(d > 1e-4).sum()} sites differ"


def test_philox_chain_bond_correlation(asd):
    """Open chain with in-kernel Philox: <S_i.S_i+1> = -(coth(bJ) - 1/(bJ))."""
    n, S = 256, 32
    lat = synth.open_chain(n, J=1.0)
    sysm = asd.System(lat)
    sp = torch.from_numpy(synth.random_unit(S * n, 2).reshape(S, n, 3)).cuda()
    sysm.thermalize(sp, 1.0, 500, asd.ASD_METROPOLIS, seed=23081, counter=0)
    acc = []
    for k in range(40):
        sysm.thermalize(sp, 1.0, 10, asd.ASD_METROPOLIS, seed=23081, counter=1000 + 10 * k)
        y = sp.double()
        acc.append((y[:, :-1] * y[:, 1:]).sum(-1).mean().item())
    ref = -(1 / math.tanh(1.0) - 1.0)
    assert abs(np.mean(acc) - ref) < 0.01, (np.mean(acc), ref)


def test_heatbath_chain_bond_correlation(asd):
    n, S, bJ = 256, 32, 2.0
    lat = synth.open_chain(n, J=1.0)
    sysm = asd.System(lat)
    sp = torch.from_numpy(synth.random_unit(S * n, 3).reshape(S, n, 3)).cuda()
    sysm.thermalize(sp, 1.0 / bJ, 200, asd.ASD_HEATBATH, seed=7)
    acc = []
    for k in range(40):
        sysm.thermalize(sp, 1.0 / bJ, 5, asd.ASD_HEATBATH, seed=7, counter=500 + 5 * k)
        y = sp.double()
        acc.append((y[:, :-1] * y[:, 1:]).sum(-1).mean().item())
    ref = -(1 / math.tanh(bJ) - 1 / bJ)
    assert abs(np.mean(acc) - ref) < 0.01, (np.mean(acc), ref)


def test_adaptive_cone_keeps_acceptance(asd):
    """At low temperature the cone shrinks until the acceptance is at least 20 %."""
    lat = synth.hypercubic(32, 2, True, J=-1.0)
    sp = torch.from_numpy(synth.random_unit(lat.n_sites, 1)[None]).cuda()
    sysm = asd.System(lat)
    sysm.thermalize(sp, 0.05, 200, asd.ASD_METROPOLIS, cone=0.0, adapt=True, seed=11)
    prop, acc, cone = sysm.thermalize(sp, 0.05, 50, asd.ASD_METROPOLIS, cone=0.3, adapt=True,
                                      seed=11, counter=200, stats=True)
    assert acc / prop >= 0.2 and 0 < cone < 1.0


def test_ll_with_dm_and_anisotropy_matches_fp64_rk4(asd):
    """All terms of Eq. 1 (exchange, bulk DM, single-ion anisotropy, field)."""
    lat = synth.with_dm_anisotropy(synth.hypercubic(8, 3, True, J=-1.0, Hz=0.3), D=0.4, A=0.7)
    S, F, stride = 2, 31, 2
    s0 = synth.random_unit(S * lat.n_sites, 13).reshape(S, lat.n_sites, 3)
    ref = dyn.ll_rk4(s0.astype(np.float64), lat.nbr, lat.J, lat.Hz, 0.01, F, stride,
                     D=lat.D, A=lat.A)
    traj = torch.zeros((lat.n_sites, S, F, 3), dtype=torch.float32, device="cuda")
    asd.System(lat).ll_integrate(torch.from_numpy(s0).cuda(), 0.01, F, stride, traj)
    assert asd.sync_status() == 0
    assert np.abs(traj.cpu().numpy() - ref).max() < 2e-5


@pytest.mark.parametrize("proposal", ["metropolis", "heatbath"])
def test_mc_with_dm_and_anisotropy_matches_oracle(asd, proposal):
    lat = synth.with_dm_anisotropy(synth.hypercubic(10, 2, True, J=1.0, Hz=0.2), D=0.5, A=0.8)
    S, sweeps, T = 2, 3, 0.7
    g = np.random.default_rng(6)
    u = g.random((sweeps, S, lat.n_sites, 4)).astype(np.float32)
    u[..., :2] = 1.0 - u[..., :2]
    s0 = synth.random_unit(S * lat.n_sites, 10).reshape(S, lat.n_sites, 3)
    Y = s0.astype(np.float64)
    for k in range(sweeps):
        Y, _, _ = dyn.mc_sweep(Y, lat.nbr, lat.J, lat.Hz, T, u[k].astype(np.float64), lat.colors,
                               proposal, D=lat.D, A=lat.A)
    sp = torch.from_numpy(s0.copy()).cuda()
    pid = asd.ASD_HEATBATH if proposal == "heatbath" else asd.ASD_METROPOLIS
    asd.System(lat).thermalize(sp, T, sweeps, pid, uniforms=torch.from_numpy(u).cuda())
    assert asd.sync_status() == 0
    d = np.abs(sp.cpu().numpy() - Y).max(-1)
    assert (d > 1e-4).mean() == 0.0, f"{(d > 1e-4).sum()} sites differ"
