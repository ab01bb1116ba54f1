"""S(q, omega) on the GPU (asd_sq_omega): parity with the FP64 definition, and the whole
chain -- LL dynamics, separable S(q,t), S(q, omega) -- against the linear spin-wave
dispersion of the paper's ferromagnetic demo model (J = -1, Hz = 0.5)."""
import numpy as np
import pytest
import torch

from oracle import spectra
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


@pytest.mark.parametrize("kind", ["none", "hann", "gauss"])
def test_transform_matches_definition(asd, kind):
    g = np.random.default_rng(4)
    S = g.standard_normal((777, 5))
    omega = np.linspace(0.0, 30.0, 301)
    out = torch.zeros((301, 5), dtype=torch.float64, device="cuda")
    asd.sq_omega(torch.from_numpy(S).cuda(), 0.02, torch.from_numpy(omega).cuda(), out,
                 window=kind, width=0.3)
    assert asd.sync_status() == 0
    ref = spectra.sq_omega(S, 0.02, omega, kind=kind, width=0.3)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_ferromagnet_spin_wave_peaks(asd):
    L, T0, n_t, dt = 32, 256, 2048, 0.01
    F = T0 + n_t - 1
    lat = synth.hypercubic(L, 2, True, J=-1.0, Hz=0.5)
    g = np.random.default_rng(11)
    Y = np.zeros((1, lat.n_sites, 3), np.float32)
    Y[0, :, :2] = 0.05 * g.standard_normal((lat.n_sites, 2))
    Y[0, :, 2] = 1.0
    Y /= np.linalg.norm(Y, axis=2, keepdims=True)
    sysm = asd.System(lat)
    traj = torch.empty((lat.n_sites, 1, F, 3), dtype=torch.float32, device="cuda")
    sysm.ll_integrate(torch.from_numpy(Y).cuda(), dt, F, 1, traj)
    q = synth.q_path_square(L)[1:]                      # q = 0 holds the static moment
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, 1.0, 0, q=q)
    Sq = torch.zeros((n_t, len(q)), dtype=torch.float64, device="cuda")
    plan.sq_separable(traj, Sq)
    omega = np.arange(0.0, 10.0, 0.01)
    Sw = torch.zeros((len(omega), len(q)), dtype=torch.float64, device="cuda")
    asd.sq_omega(Sq, dt, torch.from_numpy(omega).cuda(), Sw, window="hann")
    assert asd.sync_status() == 0
    plan.close()
    spec = Sw.cpu().numpy()
    peak = omega[np.argmax(spec, axis=0)]
    want = spectra.spin_wave_omega_square(q[:, :2])
    # Hann resolution at T = n_t dt = 20.48: main-lobe half width 2 pi / T = 0.31
    assert np.abs(peak - want).max() < 0.1, np.c_[peak, want]
