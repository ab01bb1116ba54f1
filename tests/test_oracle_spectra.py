"""Pins of the S(q, omega) oracle: closed forms of the transform, and the spin-wave
frequency against a direct integration of the linearised LL equation."""
import numpy as np

from oracle import dynamics, spectra
from paper_2308_07487_gb300 import synth


def test_delta_is_flat():
    S = np.zeros((50, 2))
    S[0] = [3.0, -1.0]
    out = spectra.sq_omega(S, 0.1, np.linspace(0, 20, 7), kind="none")
    np.testing.assert_allclose(out, np.tile([0.3, -0.1], (7, 1)), rtol=0, atol=1e-15)


def test_cosine_on_the_grid_peaks_with_closed_form_height():
    """S(t) = cos(w0 t dt), 2 w0 dt = 2 pi m / n: the value at w0 is dt (n - 1) exactly
    (1 + 2 sum cos^2 = n + sum_{t=1}^{n-1} cos(2 pi m t / n) = n - 1)."""
    n, dt, m = 64, 0.05, 5
    w0 = np.pi * m / (n * dt)
    t = np.arange(n)
    S = np.cos(w0 * t * dt)[:, None]
    val = spectra.sq_omega(S, dt, [w0], kind="none")[0, 0]
    assert abs(val - dt * (n - 1)) < 1e-12
    grid = np.linspace(0.0, 2 * w0, 401)
    spec = spectra.sq_omega(S, dt, grid, kind="hann")[:, 0]
    assert abs(grid[np.argmax(spec)] - w0) <= grid[1] - grid[0]


def test_hann_window_of_a_constant_at_zero_frequency():
    """S(t) = 1, w = 0: dt (1 + sum_{t=1}^{n-1} (1 + cos(pi t / n))) = dt n exactly, the
    cosines cancelling in pairs t <-> n - t."""
    for n in (7, 64, 301):
        val = spectra.sq_omega(np.ones((n, 1)), 0.02, [0.0], kind="hann")[0, 0]
        assert abs(val - 0.02 * n) < 1e-12 * n


def test_gaussian_window_of_a_constant_is_a_gaussian_in_frequency():
    """S(t) = 1 with the Gaussian window of width sigma = width * n_t (decayed long before
    n_t): the transform is dt sum_{t in Z} exp(-t^2 / (2 sigma^2)) cos(w t dt), which by
    Poisson summation is dt sigma sqrt(2 pi) exp(-sigma^2 (w dt)^2 / 2) for |w dt| < pi
    (the aliased terms are below exp(-2 pi^2 sigma^2 (1 - |w dt| / pi)^2), i.e. zero here)."""
    n, dt, width = 2000, 0.01, 0.05
    sigma = width * n
    omega = np.array([0.0, 0.5, 1.0, 2.0, 3.0])
    got = spectra.sq_omega(np.ones((n, 1)), dt, omega, kind="gauss", width=width)[:, 0]
    want = dt * sigma * np.sqrt(2 * np.pi) * np.exp(-0.5 * (sigma * omega * dt) ** 2)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_spin_wave_frequency_matches_linearised_ll():
    """A single plane-wave deviation on a 16^2 ferromagnet (J = -1, Hz = 0.5) integrated
    with the oracle's RK4 precesses at w(q) = Hz + 4 - 2 cos qx - 2 cos qy."""
    L = 16
    lat = synth.hypercubic(L, 2, True, J=-1.0, Hz=0.5)
    qv = np.array([2 * np.pi * 3 / L, 2 * np.pi * 1 / L])
    ph = lat.coords[:, :2] @ qv
    eps = 1e-4
    Y = np.zeros((1, lat.n_sites, 3))
    Y[0, :, 0] = eps * np.cos(ph)
    Y[0, :, 1] = eps * np.sin(ph)
    Y[0, :, 2] = 1.0
    Y /= np.linalg.norm(Y, axis=2, keepdims=True)
    dt, steps = 0.01, 100                      # w t < pi: no phase wrap
    tr = dynamics.ll_rk4(Y, lat.nbr, lat.J, 0.5, dt, steps + 1)   # [N][1][F][3]
    Yt = tr[:, 0, -1]
    # phase advance of the transverse components, averaged over the sites
    a0 = np.angle(Y[0, :, 0] + 1j * Y[0, :, 1])
    a1 = np.angle(Yt[:, 0] + 1j * Yt[:, 1])
    dphi = np.angle(np.exp(1j * (a1 - a0))).mean()
    w = abs(dphi) / (steps * dt)
    assert abs(w - spectra.spin_wave_omega_square(qv)[0]) < 1e-3
