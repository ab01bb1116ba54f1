"""FP64 oracle of the trajectory producers (test infrastructure only).

* ll_rk4           Eq. 2, dS_i/dt = (dH/dS_i) x S_i, with H of Eq. 1 (exchange, DM,
                   single-ion anisotropy, field), integrated by classic RK4 without
                   renormalisation (Section 3.1).
* mc_sweep         Section 2.1: single-spin Metropolis with trial spins uniform on the sphere
                   or in a cone about the current spin, accepted with min(1, e^{-beta dE});
                   heat-bath: the exact conditional of the terms linear in S_i, a von
                   Mises-Fisher law about -h, with a Metropolis-Hastings correction
                   min(1, e^{beta A (Sz_new^2 - Sz_old^2)}) for the anisotropy.
                   Checkerboard order: all sites of one colour, then the next.  Random
                   numbers are passed in (4 uniforms per site per sweep).
* energy, vmf_w    helpers with their closed forms pinned in tests/test_oracle_dynamics.py
"""
from __future__ import annotations

import numpy as np


def local_field(Y, nbr, J, Hz, D=None, A=0.0):
    """h_i = dH/dS_i of Eq. 1 for Y [S][N][3]:
    sum_j J_ij S_j + sum_j D_ij x S_j - 2 A S^z_i z^ - Hz z^, where D_ij is the DM vector of
    the directed bond (i, j) = slot k of site i (D_ji = -D_ij)."""
    Y = np.asarray(Y, np.float64)
    h = np.zeros_like(Y)
    for k in range(nbr.shape[1]):
        j = nbr[:, k]
        ok = j >= 0
        h[:, ok] += J[ok, k][None, :, None] * Y[:, j[ok]]
        if D is not None:
            h[:, ok] += np.cross(np.asarray(D, np.float64)[ok, k][None], Y[:, j[ok]])
    h[..., 2] -= 2.0 * A * Y[..., 2]
    h[..., 2] -= Hz
    return h


def ll_rhs(Y, nbr, J, Hz, D=None, A=0.0):
    return np.cross(local_field(Y, nbr, J, Hz, D, A), Y)


def ll_rk4(spins0, nbr, J, Hz, dt, n_frames, stride=1, D=None, A=0.0):
    """spins0 [S][N][3] -> trajectory [N][S][F][3] (FP64); frame 0 is spins0."""
    Y = np.array(spins0, np.float64)
    S, N, _ = Y.shape
    out = np.zeros((N, S, n_frames, 3))
    out[:, :, 0] = np.transpose(Y, (1, 0, 2))
    for f in range(1, n_frames):
        for _ in range(stride):
            k1 = ll_rhs(Y, nbr, J, Hz, D, A)
            k2 = ll_rhs(Y + 0.5 * dt * k1, nbr, J, Hz, D, A)
            k3 = ll_rhs(Y + 0.5 * dt * k2, nbr, J, Hz, D, A)
            k4 = ll_rhs(Y + dt * k3, nbr, J, Hz, D, A)
            Y = Y + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        out[:, :, f] = np.transpose(Y, (1, 0, 2))
    return out


def energy(Y, nbr, J, Hz, D=None, A=0.0):
    """H of Eq. 1 per sample, summed directly over the bonds (not through local_field):
    every bond appears in both neighbour lists, so each orientation carries half of
    J S_i.S_j - D_ij.(S_i x S_j) (the two orientations are equal since D_ji = -D_ij);
    then -A sum (S^z)^2 - Hz sum S^z."""
    Y = np.asarray(Y, np.float64)
    E = np.zeros(Y.shape[0])
    for k in range(nbr.shape[1]):
        j = nbr[:, k]
        ok = np.nonzero(j >= 0)[0]
        Si, Sj = Y[:, ok], Y[:, j[ok]]
        E += 0.5 * (J[ok, k][None, :] * (Si * Sj).sum(-1)).sum(-1)
        if D is not None:
            Dk = np.asarray(D, np.float64)[ok, k][None]
            E -= 0.5 * (Dk * np.cross(Si, Sj)).sum(axis=(1, 2))
    return E - A * (Y[..., 2] ** 2).sum(axis=1) - Hz * Y[..., 2].sum(axis=1)


def frame_of(m):
    """Unit vectors e1, e2 with (e1, e2, m) right-handed: e1 = normalise(a x m) with
    a = z^ when |m_z| < 0.9, else x^; e2 = m x e1."""
    m = np.asarray(m, np.float64)
    a = np.zeros_like(m)
    use_z = np.abs(m[..., 2]) < 0.9
    a[use_z, 2] = 1.0
    a[~use_z, 0] = 1.0
    e1 = np.cross(a, m)
    e1 /= np.linalg.norm(e1, axis=-1, keepdims=True)
    e2 = np.cross(m, e1)
    return e1, e2


def around(m, c, phi):
    """Unit vector at cosine c from m, azimuth phi in the frame_of(m) basis."""
    e1, e2 = frame_of(m)
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    return (c[..., None] * m + s[..., None] * (np.cos(phi)[..., None] * e1 +
                                               np.sin(phi)[..., None] * e2))


def vmf_w(kappa, u):
    """Cosine to the mean of a 3D von Mises-Fisher draw from u in (0,1] (inverse CDF)."""
    kappa = np.asarray(kappa, np.float64)
    u = np.asarray(u, np.float64)
    small = kappa < 1e-6
    ks = np.where(small, 1.0, kappa)
    w = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * ks)) / ks
    return np.where(small, 1.0 - 2.0 * u, np.maximum(-1.0, w))


def mc_sweep(Y, nbr, J, Hz, T, uniforms, colors, proposal="metropolis", cone=0.0, D=None,
             A=0.0):
    """One checkerboard sweep.  Y [S][N][3] (updated copy returned), uniforms [S][N][4].
    Returns (Y_new, accepted_count, proposed_count).  The energy change of moving S_i is
    (S' - S).h_lin - A (S'z^2 - Sz^2), h_lin the field of the terms linear in S_i."""
    Y = np.array(Y, np.float64)
    beta = 1.0 / T
    acc_total = 0
    prop_total = 0
    for sites in colors:
        u = uniforms[:, sites]                       # [S][n][4]
        # neighbours are of other colours; the anisotropy term is kept apart
        h = local_field(Y, nbr, J, Hz, D, 0.0)[:, sites]
        old = Y[:, sites]
        if proposal == "heatbath":
            hn = np.linalg.norm(h, axis=-1)
            m = np.where(hn[..., None] > 0, -h / np.where(hn > 0, hn, 1.0)[..., None],
                         np.array([0.0, 0.0, 1.0]))
            new = around(m, vmf_w(beta * hn, u[..., 0]), 2 * np.pi * u[..., 1])
            la = beta * A * (new[..., 2] ** 2 - old[..., 2] ** 2)
            accept = (la >= 0) | (u[..., 2] < np.exp(np.minimum(la, 0.0)))
        else:
            cmin = -1.0 if (cone <= 0 or cone >= np.pi) else np.cos(cone)
            new = around(old, 1.0 - u[..., 0] * (1.0 - cmin), 2 * np.pi * u[..., 1])
            dE = ((new - old) * h).sum(-1) - A * (new[..., 2] ** 2 - old[..., 2] ** 2)
            la = -beta * dE
            accept = (la >= 0) | (u[..., 2] < np.exp(np.minimum(la, 0.0)))
        Y[:, sites] = np.where(accept[..., None], new, old)
        acc_total += int(accept.sum())
        prop_total += accept.size
    return Y, acc_total, prop_total
