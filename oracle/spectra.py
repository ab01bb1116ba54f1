"""S(q, omega) from S(q, t) by the windowed cosine transform (Section 4), written out in FP64.

Test infrastructure only (the GPU path is asd_sq_omega).  With the even extension
S(q, -t) = S(q, t):
    S(q, w) = dt * ( v_0 S(q, 0) + 2 sum_{t=1}^{n_t-1} v_t S(q, t) cos(w t dt) )
with v_t = 1, the Hann taper (1 + cos(pi t / n_t)) / 2, or the Gaussian
exp(-(t / (width n_t))^2 / 2)."""
from __future__ import annotations

import numpy as np


def window(n_t, kind="hann", width=0.25):
    t = np.arange(n_t, dtype=np.float64)
    if kind == "none":
        return np.ones(n_t)
    if kind == "hann":
        return 0.5 * (1.0 + np.cos(np.pi * t / n_t))
    if kind == "gauss":
        return np.exp(-0.5 * (t / (width * n_t)) ** 2)
    raise ValueError(kind)


def sq_omega(S, dt, omega, kind="hann", width=0.25):
    """S [n_t][n_q] -> [n_w][n_q]."""
    S = np.asarray(S, np.float64)
    n_t = S.shape[0]
    v = window(n_t, kind, width)
    t = np.arange(n_t, dtype=np.float64)
    out = np.zeros((len(omega), S.shape[1]))
    for k, w in enumerate(np.asarray(omega, np.float64)):
        c = np.cos(w * t * dt)
        c[1:] *= 2.0
        out[k] = dt * ((v * c)[:, None] * S).sum(axis=0)
    return out


def spin_wave_omega_square(q, J=-1.0, Hz=0.5):
    """Linear spin-wave frequency of the LL equation dS/dt = (dH/dS) x S on a square
    lattice with H = J sum_<ij> S_i.S_j - Hz sum_i S^z_i, J < 0 (ferromagnet along +z):
    small deviations d_i obey dd_i/dt = z^ x (|J| sum_j d_j - (4|J| + Hz) d_i), so a plane
    wave precesses at w(q) = Hz + |J| (4 - 2 cos qx - 2 cos qy)."""
    q = np.atleast_2d(q)
    return Hz + abs(J) * (4.0 - 2.0 * np.cos(q[:, 0]) - 2.0 * np.cos(q[:, 1]))
