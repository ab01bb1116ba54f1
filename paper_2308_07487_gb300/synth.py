"""Seeded synthetic inputs: lattices, couplings, positions, spins, trajectories, q-vectors.

This module only *generates inputs*.  It holds none of the correlation method's
arithmetic (no distance bins, no pair sums, no dynamics), so both the CUDA path and
the FP64 oracle can be fed from it without sharing any part of the computation.

Workload recipes follow the systems the paper studies: classical Heisenberg spins
on square / simple-cubic lattices with nearest-neighbour exchange (Section 2, Eq. 1;
Section 3 uses the 2D square lattice), plus the non-periodic jittered +-J glass and
batched ensembles used to exercise the non-periodic and batched paths.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2308  # every workload seed is 2308<k>


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


@dataclass
class Lattice:
    """A classical spin system on N sites.

    coords  int32 [N,3]  integer lattice coordinates (unused axes are 0)
    L       (Lx,Ly,Lz)   extents (1 for unused axes)
    periodic             minimum-image distances / wrapped neighbours
    nbr     int32 [N,z]  neighbour site per slot, -1 where absent
    J       f32   [N,z]  coupling per slot (0 where absent); J_ij == J_ji
    pos     f32   [N,3]  Cartesian positions (coords, or jittered coords)
    colors  list of int32 arrays: sites of each checkerboard colour
    D, A    optional DM vectors per directed bond and single-ion anisotropy (Eq. 1 terms)
    """
    dim: int
    L: tuple
    periodic: bool
    coords: np.ndarray
    nbr: np.ndarray
    J: np.ndarray
    pos: np.ndarray
    colors: list = field(default_factory=list)
    Hz: float = 0.0
    D: np.ndarray | None = None   # f32 [N,z,3] DM vector per directed bond (D_ji = -D_ij)
    A: float = 0.0                # single-ion anisotropy

    @property
    def n_sites(self) -> int:
        return int(self.coords.shape[0])


def _site_order(L, block):
    """Enumerate lattice points; with `block`, sites are numbered block by block
    (x fastest inside a block, blocks in x-fastest order)."""
    Lx, Ly, Lz = L
    if block is None:
        z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
        return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)
    bx, by, bz = block
    assert Lx % bx == 0 and Ly % by == 0 and Lz % bz == 0
    out = []
    for BZ in range(Lz // bz):
        for BY in range(Ly // by):
            for BX in range(Lx // bx):
                z, y, x = np.meshgrid(np.arange(bz) + BZ * bz, np.arange(by) + BY * by,
                                      np.arange(bx) + BX * bx, indexing="ij")
                out.append(np.stack([x.ravel(), y.ravel(), z.ravel()], 1))
    return np.concatenate(out).astype(np.int32)


def hypercubic(L: int, dim: int, periodic: bool = True, J: float = 1.0, Hz: float = 0.0,
               pm_j: bool = False, p: float = 0.5, seed: int = 0, block=None,
               jitter: float = 0.0) -> Lattice:
    """Square (dim=2) or simple-cubic (dim=3) lattice of side L with nearest-neighbour
    coupling J (Eq. 1 sign convention: J>0 antiferromagnetic, J<0 ferromagnetic), or
    random +-J couplings with probability p of +J.  `jitter` adds N(0, jitter^2) to
    every Cartesian coordinate (the non-periodic glass recipe)."""
    Ls = (L, L, L if dim == 3 else 1)
    coords = _site_order(Ls, block)
    N = coords.shape[0]
    index = np.full(Ls[::-1], -1, dtype=np.int64)  # [z][y][x] -> site
    index[coords[:, 2], coords[:, 1], coords[:, 0]] = np.arange(N)
    z_nb = 2 * dim
    nbr = np.full((N, z_nb), -1, dtype=np.int32)
    for a in range(dim):
        for sgn_i, sgn in enumerate((+1, -1)):
            c = coords.astype(np.int64).copy()
            c[:, a] += sgn
            if periodic:
                c[:, a] %= Ls[a]
                ok = np.ones(N, bool)
            else:
                ok = (c[:, a] >= 0) & (c[:, a] < Ls[a])
                c[:, a] = np.clip(c[:, a], 0, Ls[a] - 1)
            nb = index[c[:, 2], c[:, 1], c[:, 0]]
            nbr[:, 2 * a + sgn_i] = np.where(ok, nb, -1)
    Jt = np.zeros((N, z_nb), dtype=np.float32)
    if pm_j:
        g = rng(seed)
        # one draw per undirected bond, stored on both ends
        for a in range(dim):
            draw = np.where(g.random(N) < p, 1.0, -1.0).astype(np.float32)
            fwd = nbr[:, 2 * a]
            ok = fwd >= 0
            Jt[ok, 2 * a] = draw[ok]
            Jt[fwd[ok], 2 * a + 1] = draw[ok]
    else:
        Jt[nbr >= 0] = J
    pos = coords.astype(np.float32)
    if jitter > 0:
        pos = (coords.astype(np.float64) + rng(seed + 1).normal(0.0, jitter, size=(N, 3))).astype(np.float32)
        if dim == 2:
            pos[:, 2] = 0.0
    parity = coords.sum(1) % 2
    colors = [np.nonzero(parity == c)[0].astype(np.int32) for c in (0, 1)]
    return Lattice(dim=dim, L=Ls, periodic=periodic, coords=coords, nbr=nbr, J=Jt,
                   pos=pos, colors=colors, Hz=Hz)


def open_chain(N: int, J: float = 1.0) -> Lattice:
    """Open 1D chain (bond angles are independent: a closed-form MC check)."""
    coords = np.zeros((N, 3), np.int32)
    coords[:, 0] = np.arange(N)
    nbr = np.full((N, 2), -1, np.int32)
    nbr[1:, 1] = np.arange(N - 1)
    nbr[:-1, 0] = np.arange(1, N)
    Jt = np.where(nbr >= 0, J, 0.0).astype(np.float32)
    colors = [np.arange(0, N, 2, dtype=np.int32), np.arange(1, N, 2, dtype=np.int32)]
    return Lattice(dim=1, L=(N, 1, 1), periodic=False, coords=coords, nbr=nbr, J=Jt,
                   pos=coords.astype(np.float32), colors=colors)


def random_unit(n: int, seed: int) -> np.ndarray:
    """n i.i.d. unit vectors, uniform on the sphere, FP32 [n,3]."""
    v = rng(seed).normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


def traj_iid(N: int, F: int, seed: int, S: int = 1) -> np.ndarray:
    """I.i.d. random unit spins in every frame: trajectory [N][S][F][3] FP32 (the
    worst case for cancellation: no correlation beyond the self pair at t=0)."""
    return random_unit(N * S * F, seed).reshape(N, S, F, 3)


def traj_precess(N: int, F: int, seed: int, S: int = 1, order: float = 0.6,
                 omega: float = 0.05) -> np.ndarray:
    """Correlated synthetic trajectory [N][S][F][3] FP32: unit spins tilted towards a
    common axis (weight `order`) that precess about z with site-dependent rates, so
    C(r,t) has structure in both r and t."""
    g = rng(seed)
    base = g.normal(size=(N * S, 3))
    base /= np.linalg.norm(base, axis=1, keepdims=True)
    axis = np.array([0.3, 0.2, 0.93])
    axis /= np.linalg.norm(axis)
    s0 = order * axis + (1.0 - order) * base
    s0 /= np.linalg.norm(s0, axis=1, keepdims=True)
    w = omega * (1.0 + 0.5 * g.standard_normal(N * S))
    f = np.arange(F)
    ang = w[:, None] * f[None, :]
    c, s = np.cos(ang), np.sin(ang)
    x = c * s0[:, 0:1] - s * s0[:, 1:2]
    y = s * s0[:, 0:1] + c * s0[:, 1:2]
    z = np.broadcast_to(s0[:, 2:3], x.shape)
    tr = np.stack([x, y, z], -1).reshape(N, S, F, 3)
    return tr.astype(np.float32)


def traj_static(N: int, F: int, direction=(0.0, 0.0, 1.0), S: int = 1) -> np.ndarray:
    """Every spin equal to one unit vector in every frame (a ferromagnetic ground state)."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    return np.broadcast_to(d.astype(np.float32), (N, S, F, 3)).copy()


def q_vectors_glass(seed: int = SEED_BASE * 10 + 3, n_mag: int = 16) -> np.ndarray:
    """64 q-vectors: directions (100), (110), (111) and one seeded random direction,
    each with magnitudes pi*m/16, m = 0..15.  FP64 [64,3]."""
    dirs = [np.array([1.0, 0, 0]), np.array([1.0, 1, 0]) / math.sqrt(2),
            np.array([1.0, 1, 1]) / math.sqrt(3)]
    r = rng(seed).normal(size=3)
    dirs.append(r / np.linalg.norm(r))
    mags = math.pi * np.arange(n_mag) / 16.0
    return np.array([d * m for d in dirs for m in mags], np.float64)


def q_path_square(L: int) -> np.ndarray:
    """Reciprocal-lattice vectors of an LxL square lattice along (0,0)->(pi,0)->(pi,pi)->(0,0)."""
    h = L // 2
    pts = [(k, 0) for k in range(0, h)] + [(h, k) for k in range(0, h)] + \
          [(k, k) for k in range(h, 0, -1)]
    return np.array([[2 * math.pi * a / L, 2 * math.pi * b / L, 0.0] for a, b in pts], np.float64)


# ---------------------------------------------------------------------------------
# Workload configurations (the sizes of the paper-style runs)
# ---------------------------------------------------------------------------------

@dataclass
class CorrConfig:
    name: str
    lattice: Lattice
    F: int
    T0: int
    n_t: int
    w: float
    n_bins: int
    S: int = 1
    q: np.ndarray | None = None
    T: float = 1.0
    seed: int = 0


def cfg_small_2d() -> CorrConfig:
    """16x16 periodic square lattice, N=256, J=+1, T=0.5, F=96, T0=64, 32
    displacements, bins of width 1 (12 bins cover the largest minimum-image distance)."""
    lat = hypercubic(16, 2, True, J=1.0, seed=SEED_BASE * 10 + 1)
    return CorrConfig("sq16_periodic_N256", lat, F=96, T0=64, n_t=32, w=1.0, n_bins=12,
                      T=0.5, seed=SEED_BASE * 10 + 1)


def cfg_cubic40() -> CorrConfig:
    """40^3 periodic simple-cubic lattice, N=64000, J=+1, T=1.2, F=1200, T0=1000,
    200 displacements, shell bins of width 0.5 (70 bins)."""
    lat = hypercubic(40, 3, True, J=1.0, seed=SEED_BASE * 10 + 2)
    return CorrConfig("sc40_periodic_N64000", lat, F=1200, T0=1000, n_t=200, w=0.5,
                      n_bins=70, T=1.2, seed=SEED_BASE * 10 + 2)


def cfg_glass64(block=(4, 4, 8)) -> CorrConfig:
    """64^3 = 262144 sites at jittered (sigma=0.1) simple-cubic positions, open
    boundaries, +-J couplings (p=0.5), numbered in 4x4x8 spatial blocks; F=640,
    T0=512, 128 displacements, 256 bins of width 0.5, 64 q-vectors."""
    s = SEED_BASE * 10 + 3
    lat = hypercubic(64, 3, False, pm_j=True, p=0.5, seed=s, block=block, jitter=0.1)
    return CorrConfig("glass64_open_N262144", lat, F=640, T0=512, n_t=128, w=0.5,
                      n_bins=256, q=q_vectors_glass(), T=1.0, seed=s)


def ensemble_sizes(n: int = 96, seed: int = SEED_BASE * 10 + 4, lo: int = 1024, hi: int = 40000):
    """Uneven ensemble: N_s log-uniform in [lo, hi], dimension alternating 2/3 (seeded
    order), L = round(N_s^(1/d)), N_s := L^d."""
    g = rng(seed)
    out = []
    dims = g.permutation(np.array([2, 3] * (n // 2) + [2] * (n % 2)))
    for k in range(n):
        Ns = math.exp(g.uniform(math.log(lo), math.log(hi)))
        d = int(dims[k])
        L = max(2, int(round(Ns ** (1.0 / d))))
        out.append((d, L))
    return out


def with_dm_anisotropy(lat: Lattice, D: float = 0.0, A: float = 0.0) -> Lattice:
    """A copy of `lat` with bulk-type DM vectors D_ij = D * (unit bond vector from i to j,
    minimum image when periodic; antisymmetric by construction) and anisotropy A."""
    import dataclasses
    N, z = lat.nbr.shape
    Dv = np.zeros((N, z, 3), np.float32)
    Ls = np.array(lat.L, np.float64)
    for k in range(z):
        j = lat.nbr[:, k]
        ok = j >= 0
        d = lat.coords[j[ok]].astype(np.float64) - lat.coords[ok].astype(np.float64)
        if lat.periodic:
            d -= Ls * np.round(d / Ls)
        n = np.linalg.norm(d, axis=1, keepdims=True)
        Dv[ok, k] = (D * d / np.where(n > 0, n, 1.0)).astype(np.float32)
    return dataclasses.replace(lat, D=Dv, A=float(A))
