"""Independent restatements used only to pin the loop oracle (test infrastructure).

Nothing here shares code with paircorr_ref.c: the distance bins are recomputed
from a threshold table, and the pair sums are obtained by different algorithms:

* lattice_fft_corr  -- on (periodic or open) lattices the ordered-pair sum over a
  bin equals a sum over displacement vectors d of the lattice cross-correlation
  X_d(t) = sum_i sum_{s,t0,a} S_{i,a}(t0+t) S_{i+d,a}(t0), evaluated with FFTs in
  space and time (FP64).  This is the momentum-space route the paper mentions for
  periodic lattices (Section 1, Section 3 opening paragraph).
* separable_phase_sum -- the phase form of Eq. 3 with Eq. 6 factorises through
  cos(a-b) = cos a cos b + sin a sin b into per-site transforms
  F^c(q,f) = sum_i cos(q.r_i) S_i(f), F^s likewise (a non-uniform DFT), so
  sum_ij cos(q.(r_i-r_j)) G_ij(t) = sum_{s,t0,a} F^c(t0+t) F^c(t0) + F^s(t0+t) F^s(t0).
"""
from __future__ import annotations

import numpy as np


def bins_from_thresholds(d2, w, n_bins):
    """bin = number of k in 1..n_bins with (k w)^2 <= d2 (>= n_bins means dropped)."""
    thr = (np.arange(1, n_bins + 1, dtype=np.float64) * w) ** 2
    return np.searchsorted(thr, np.asarray(d2, np.float64), side="right")


def lattice_fft_corr(traj, T0, t_list, coords, L, periodic, w, n_bins):
    """Binned C_sum[t][b] on a full lattice via FFT cross-correlation (FP64)."""
    tr = np.asarray(traj, np.float64)
    if tr.ndim == 3:
        tr = tr[:, None]
    N, S, F, _ = tr.shape
    Lx, Ly, Lz = (int(v) for v in L)
    assert N == Lx * Ly * Lz, "FFT check needs every lattice point occupied"
    pad = (Lz, Ly, Lx) if periodic else tuple(2 * v if v > 1 else 1 for v in (Lz, Ly, Lx))
    t_list = np.atleast_1d(t_list)
    nf = 1
    while nf < F + T0:
        nf *= 2
    V = pad[0] * pad[1] * pad[2]
    # Yhat[t](k) = sum_{s,t0,a} G_k(t0+t) conj(G_k(t0)), accumulated one (sample, component)
    # and one chunk of wave vectors at a time (bounded memory at any lattice size)
    Yhat = np.zeros((len(t_list), V), np.complex128)
    chunk = max(1, (1 << 25) // (nf * 16))
    for s in range(S):
        for a in range(3):
            g = np.zeros((F,) + tuple(int(v) for v in (Lz, Ly, Lx)), np.float64)
            g[:, coords[:, 2], coords[:, 1], coords[:, 0]] = tr[:, s, :, a].T
            # spatial transform of every frame, flattened over k
            G = np.fft.fftn(g, s=pad, axes=(1, 2, 3)).reshape(F, V)
            del g
            for k0 in range(0, V, chunk):
                Gc = G[:, k0:k0 + chunk]
                # sum_{t0<T0} a[t0+t] conj(b[t0]) = ifft(fft(a) conj(fft(b)))[t], b = a cut at T0
                A = np.fft.fft(Gc, n=nf, axis=0)
                B = np.fft.fft(Gc[:T0], n=nf, axis=0)
                Yhat[:, k0:k0 + chunk] += np.fft.ifft(A * np.conj(B), axis=0)[t_list]
            del G
    # X_d = sum_x a(x) b(x+d) = (1/V) sum_k conj(A_k) B_k e^{ikd}: conj of the above
    X = np.fft.ifftn(np.conj(Yhat).reshape((len(t_list),) + pad), axes=(1, 2, 3)).real
    # displacement vectors of every grid offset and their squared distance
    dz, dy, dx = np.meshgrid(np.arange(pad[0]), np.arange(pad[1]), np.arange(pad[2]), indexing="ij")
    comps = []
    for d, Lv, P in ((dx, Lx, pad[2]), (dy, Ly, pad[1]), (dz, Lz, pad[0])):
        if periodic:
            comps.append(np.minimum(d, Lv - d))
        else:
            comps.append(np.where(d < P - d, d, P - d))   # signed offset magnitude for open grids
    d2 = comps[0] ** 2 + comps[1] ** 2 + comps[2] ** 2
    b = bins_from_thresholds(d2, w, n_bins)
    out = np.zeros((len(t_list), n_bins))
    for k in range(n_bins):
        m = b == k
        if m.any():
            out[:, k] = X[:, m].sum(axis=1)
    return out


def separable_phase_sum(traj, T0, t_list, pos, q, center=False, part="cos"):
    """Sq_sum[t][q] = sum_ij cos(q.(r_i-r_j)) G_ij(t) through the factorised transform
    (part="sin": sum_ij sin(q.(r_i-r_j)) G_ij(t) = sum F^s_A F^c_B - F^c_A F^s_B).

    F^c = C^T X and F^s = S^T X with C[i][q] = cos(q.r_i), S[i][q] = sin(q.r_i) and X the
    trajectory flattened to [N][S*F*3] (FP64 matrix products), then per t the sum over
    samples, origins and components of F(t0 + t) F(t0).  Centring (per site, over samples
    and origins, of both operands as in Eq. 5) is linear, so it is applied to the
    transforms: the transform of a centred operand is the transform minus its mean."""
    tr = np.asarray(traj, np.float64)
    if tr.ndim == 3:
        tr = tr[:, None]
    N, S, F, _ = tr.shape
    r = np.asarray(pos, np.float64)
    ph = r @ np.asarray(q, np.float64).T            # [N][n_q]
    c, s = np.cos(ph), np.sin(ph)
    X = tr.reshape(N, S * F * 3)
    Fc = (c.T @ X).reshape(-1, S, F, 3)             # [n_q][S][F][3]
    Fs = (s.T @ X).reshape(-1, S, F, 3)
    t_list = np.atleast_1d(t_list)
    out = np.zeros((len(t_list), len(q)))

    def window(Fx, t):
        w = Fx[:, :, t:t + T0]
        if center:
            w = w - w.mean(axis=(1, 2), keepdims=True)
        return w
    Bc, Bs = window(Fc, 0), window(Fs, 0)
    for k, t in enumerate(t_list):
        if part == "sin":
            out[k] = (window(Fs, t) * Bc).sum(axis=(1, 2, 3)) - (window(Fc, t) * Bs).sum(axis=(1, 2, 3))
        else:
            out[k] = (window(Fc, t) * Bc).sum(axis=(1, 2, 3)) + (window(Fs, t) * Bs).sum(axis=(1, 2, 3))
    return out


def total_moment_corr(traj, T0, t_list):
    """q = 0 closed form: sum_ij G_ij(t) = sum_{s,t0} M(t0+t) . M(t0), M = sum_i S_i."""
    tr = np.asarray(traj, np.float64)
    if tr.ndim == 3:
        tr = tr[:, None]
    M = tr.sum(axis=0)                              # [S][F][3]
    return np.array([(M[:, t:t + T0] * M[:, :T0]).sum() for t in np.atleast_1d(t_list)])
