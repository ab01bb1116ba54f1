"""Pins of the FP64 producer oracle (LL RK4, Monte Carlo) against closed forms and
invariants: single-spin precession, the exchange dimer, total-spin conservation,
energy conservation, the open-chain bond correlation -L(beta J) (uniform, cone and
heat-bath proposals), vMF moments; for the DM and anisotropy terms of Eq. 1 the
gradient of the energy, DM spiral energies and pitch, anisotropy precession, S^z
conservation with DM along z, and the sampled <(S^z)^2> of an anisotropic spin."""
import math

import numpy as np

from oracle import dynamics as dyn
from paper_2308_07487_gb300 import synth


def test_single_spin_precession_closed_form():
    """dS/dt = (-Hz z^) x S: S_x = x0 cos(Hz t) + y0 sin(Hz t), S_y = y0 cos - x0 sin."""
    nbr = np.full((1, 1), -1, np.int32)
    J = np.zeros((1, 1), np.float32)
    s0 = np.array([[[0.6, 0.0, 0.8]]])
    Hz, dt, F = 0.5, 0.01, 201
    tr = dyn.ll_rk4(s0, nbr, J, Hz, dt, F)
    t = dt * np.arange(F)
    ref = np.stack([0.6 * np.cos(Hz * t), -0.6 * np.sin(Hz * t), 0.8 * np.ones(F)], -1)
    np.testing.assert_allclose(tr[0, 0], ref, atol=1e-10)


def test_exchange_dimer_rotates_about_total_spin():
    """Two spins, H = J S1.S2: S1 rotates about M = S1 + S2 at rate J|M| (Rodrigues)."""
    nbr = np.array([[1], [0]], np.int32)
    J = np.full((2, 1), 1.3, np.float32)
    Jv = float(J[0, 0])            # the coupling the dynamics sees (FP32-rounded 1.3)
    s1 = np.array([0.0, 0.6, 0.8])
    s2 = np.array([1.0, 0.0, 0.0])
    M = s1 + s2
    k = M / np.linalg.norm(M)
    t_end = 1.5
    th = Jv * np.linalg.norm(M) * t_end
    ref = s1 * math.cos(th) + np.cross(k, s1) * math.sin(th) + k * k.dot(s1) * (1 - math.cos(th))
    errs = []
    for dt in (0.02, 0.01):
        n = int(round(t_end / dt))
        tr = dyn.ll_rk4(np.array([[s1, s2]]), nbr, J, 0.0, dt, n + 1)
        errs.append(np.abs(tr[0, 0, -1] - ref).max())
    assert errs[1] < 1e-6
    # fourth order: halving dt divides the global error by about 2^4
    assert 12 < errs[0] / errs[1] < 20, errs


def test_total_spin_conserved_and_energy_drift_small():
    lat = synth.hypercubic(6, 2, True, J=-1.0)
    s0 = synth.random_unit(lat.n_sites * 2, 7).reshape(2, lat.n_sites, 3).astype(np.float64)
    tr = dyn.ll_rk4(s0, lat.nbr, lat.J, 0.0, 0.01, 101)
    M = tr.sum(axis=0)  # [S][F][3]
    assert np.abs(M - M[:, :1]).max() < 1e-11
    Y0 = np.transpose(tr[:, :, 0], (1, 0, 2))
    Y1 = np.transpose(tr[:, :, -1], (1, 0, 2))
    e0, e1 = dyn.energy(Y0, lat.nbr, lat.J, 0.0), dyn.energy(Y1, lat.nbr, lat.J, 0.0)
    assert np.abs(e1 - e0).max() < 1e-6 * lat.n_sites


def test_field_precesses_total_moment():
    """With Hz != 0 and exchange, M(t) precesses about z at rate Hz (exchange torques cancel)."""
    lat = synth.hypercubic(4, 2, True, J=1.0)
    s0 = synth.random_unit(lat.n_sites, 3)[None].astype(np.float64)
    Hz, dt, F = 0.7, 0.01, 51
    tr = dyn.ll_rk4(s0, lat.nbr, lat.J, Hz, dt, F)
    M = tr.sum(axis=0)[0]
    t = dt * (F - 1)
    c, s = math.cos(Hz * t), math.sin(Hz * t)
    ref = np.array([M[0, 0] * c + M[0, 1] * s, M[0, 1] * c - M[0, 0] * s, M[0, 2]])
    np.testing.assert_allclose(M[-1], ref, atol=1e-8)


def test_vmf_inverse_cdf_moments():
    """E[w] = coth(kappa) - 1/kappa for the 3D von Mises-Fisher law."""
    u = (np.arange(200000) + 0.5) / 200000
    for kappa in (0.3, 2.0, 15.0):
        w = dyn.vmf_w(kappa, u)
        assert abs(w.mean() - (1 / math.tanh(kappa) - 1 / kappa)) < 1e-4


def _chain_bond_corr(proposal, T, J=1.0, n=64, sweeps=3000, seed=1, cone=0.0):
    lat = synth.open_chain(n, J=J)
    g = np.random.default_rng(seed)
    Y = synth.random_unit(n, seed)[None].astype(np.float64)
    acc = []
    for sw in range(sweeps):
        u = g.random((1, n, 4))
        u[..., :2] = 1.0 - u[..., :2]  # (0, 1]
        Y, _, _ = dyn.mc_sweep(Y, lat.nbr, lat.J, 0.0, T, u, lat.colors, proposal, cone=cone)
        if sw >= 300:
            acc.append((Y[0, :-1] * Y[0, 1:]).sum(-1).mean())
    return float(np.mean(acc))


def test_open_chain_bond_correlation_metropolis():
    """Open chain: bond angles are independent, <S_i.S_i+1> = -(coth(bJ) - 1/(bJ))."""
    bJ = 1.0
    ref = -(1 / math.tanh(bJ) - 1 / bJ)
    got = _chain_bond_corr("metropolis", 1.0)
    assert abs(got - ref) < 0.02, (got, ref)


def test_open_chain_bond_correlation_cone_proposal():
    """Metropolis with moves uniform on a cap of half-angle 0.8 about the current spin (a
    symmetric proposal: its density depends only on the angle moved) samples the same
    Boltzmann law: <S_i.S_i+1> = -(coth(bJ) - 1/(bJ)).  A cap centred anywhere but on the
    current spin fails this."""
    bJ = 1.0
    ref = -(1 / math.tanh(bJ) - 1 / bJ)
    got = _chain_bond_corr("metropolis", 1.0, cone=0.8, seed=3)
    assert abs(got - ref) < 0.02, (got, ref)


def test_open_chain_bond_correlation_heatbath():
    bJ = 2.0
    ref = -(1 / math.tanh(bJ) - 1 / bJ)
    got = _chain_bond_corr("heatbath", 0.5)
    assert abs(got - ref) < 0.02, (got, ref)


def test_frame_is_orthonormal_right_handed():
    m = synth.random_unit(50, 4).astype(np.float64)
    m[0] = [0, 0, 1]
    m[1] = [0, 0, -1]
    e1, e2 = dyn.frame_of(m)
    np.testing.assert_allclose(np.cross(e1, e2), m, atol=1e-12)
    np.testing.assert_allclose((e1 * m).sum(-1), 0, atol=1e-12)


# ---- the DM and single-ion anisotropy terms of Eq. 1 ----

def _dm_z_lattice(L=6, D=0.7, A=0.4, Hz=0.2, J=-1.0):
    """Square lattice with DM vectors along z, D_ij = D (d_ij . x^) z^ (antisymmetric), so
    H stays invariant under rotations about z."""
    lat = synth.hypercubic(L, 2, True, J=J, Hz=Hz)
    lat = synth.with_dm_anisotropy(lat, D=1.0, A=A)
    Dz = np.zeros_like(lat.D)
    Dz[..., 2] = D * lat.D[..., 0]
    return lat, Dz


def test_field_is_the_gradient_of_eq1():
    """local_field (written from the derivative) equals the finite-difference gradient of
    energy (written from Eq. 1 bond by bond), with exchange, DM, anisotropy and field."""
    lat = synth.with_dm_anisotropy(synth.hypercubic(4, 3, True, J=0.7, Hz=0.3), D=0.45, A=0.6)
    g = np.random.default_rng(3)
    Y = g.standard_normal((1, lat.n_sites, 3))
    h = dyn.local_field(Y, lat.nbr, lat.J, lat.Hz, lat.D, lat.A)
    eps = 1e-6
    for i in (0, 5, 17, 63):
        for a in range(3):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[0, i, a] += eps
            Ym[0, i, a] -= eps
            fd = (dyn.energy(Yp, lat.nbr, lat.J, lat.Hz, lat.D, lat.A) -
                  dyn.energy(Ym, lat.nbr, lat.J, lat.Hz, lat.D, lat.A))[0] / (2 * eps)
            assert abs(fd - h[0, i, a]) < 1e-6, (i, a, fd, h[0, i, a])


def test_dm_chain_spiral_energy_and_pitch():
    """Open chain along x with FM exchange J < 0 and DM vectors D z^ on the bonds i -> i+1
    (-D z^ on i+1 -> i).  For the planar spiral S_k = (cos k theta, sin k theta, 0) each bond
    contributes J cos theta - D sin theta (Eq. 1's -D_ij.(S_i x S_j) with S_i x S_i+1 =
    sin theta z^), so the spiral of lowest energy has pitch atan(D / |J|), turning
    counter-clockwise about z for D > 0 and clockwise for D < 0."""
    n, J = 24, -1.0
    lat = synth.open_chain(n, J=J)
    thetas = np.linspace(-np.pi, np.pi, 3601)
    for Dm in (0.6, -0.35):
        Dv = np.zeros((n, 2, 3))
        Dv[:-1, 0, 2] = Dm    # slot 0: bond i -> i + 1
        Dv[1:, 1, 2] = -Dm    # slot 1: bond i + 1 -> i
        k = np.arange(n)[None, :]
        Y = np.stack([np.cos(k * thetas[:, None]), np.sin(k * thetas[:, None]),
                      np.zeros((len(thetas), n))], axis=-1)
        E = dyn.energy(Y, lat.nbr, lat.J, 0.0, Dv, 0.0)
        np.testing.assert_allclose(E, (n - 1) * (J * np.cos(thetas) - Dm * np.sin(thetas)),
                                   rtol=0, atol=1e-10)
        best = thetas[np.argmin(E)]
        assert abs(best - math.atan(Dm / abs(J))) <= thetas[1] - thetas[0]


def test_anisotropy_precession_closed_form():
    """A single spin under -A (S^z)^2 only: h = -2 A S^z z^, so S^z is constant and the
    azimuth turns at -2 A S^z."""
    lat = synth.open_chain(1, J=0.0)
    A, dt, F = 1.3, 0.001, 401
    s0 = np.array([[[0.6, 0.0, 0.8]]])
    tr = dyn.ll_rk4(s0, lat.nbr, lat.J, 0.0, dt, F, A=A)[0, 0]
    t = dt * np.arange(F)
    phi = -2.0 * A * 0.8 * t
    ref = np.stack([0.6 * np.cos(phi), 0.6 * np.sin(phi), np.full(F, 0.8)], 1)
    assert np.abs(tr - ref).max() < 1e-9


def test_dm_along_z_conserves_total_sz_and_energy():
    lat, Dz = _dm_z_lattice()
    s0 = synth.random_unit(lat.n_sites, 8).reshape(1, lat.n_sites, 3).astype(np.float64)
    tr = dyn.ll_rk4(s0, lat.nbr, lat.J, lat.Hz, 0.005, 201, D=Dz, A=lat.A)
    Sz = tr[:, 0, :, 2].sum(0)
    assert np.abs(Sz - Sz[0]).max() < 1e-9
    E0 = dyn.energy(s0, lat.nbr, lat.J, lat.Hz, Dz, lat.A)[0]
    E1 = dyn.energy(np.transpose(tr[:, :, -1], (1, 0, 2)), lat.nbr, lat.J, lat.Hz, Dz, lat.A)[0]
    assert abs(E1 - E0) < 1e-8 * lat.n_sites


def _single_spin_anisotropy_chain(proposal, A=1.5, T=0.5, S=4000, sweeps=160):
    lat = synth.open_chain(1, J=0.0)
    g = np.random.default_rng(21)
    Y = synth.random_unit(S, 2).reshape(S, 1, 3).astype(np.float64)
    zz = []
    for k in range(sweeps):
        u = g.random((S, 1, 4))
        u[..., :2] = 1.0 - u[..., :2]
        Y, _, _ = dyn.mc_sweep(Y, lat.nbr, lat.J, 0.0, T, u, lat.colors, proposal, A=A)
        if k >= 40:
            zz.append(Y[:, 0, 2] ** 2)
    per_chain = np.mean(zz, axis=0)
    x = np.linspace(-1.0, 1.0, 20001)
    w = np.exp(A / T * x * x)
    exact = np.trapezoid(x * x * w, x) / np.trapezoid(w, x)
    return per_chain.mean(), per_chain.std() / np.sqrt(S), exact


def test_metropolis_samples_the_anisotropy():
    m, se, exact = _single_spin_anisotropy_chain("metropolis")
    assert abs(m - exact) < 5 * se + 1e-3, (m, se, exact)


def test_heatbath_with_correction_samples_the_anisotropy():
    m, se, exact = _single_spin_anisotropy_chain("heatbath")
    assert abs(m - exact) < 5 * se + 1e-3, (m, se, exact)
