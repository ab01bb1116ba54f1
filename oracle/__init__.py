"""FP64 CPU oracle for the spin pair correlation path (arXiv 2308.07487).

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs may import this package.  It shares no
code with the CUDA library (paper_2308_07487_gb300/csrc) and never imports it.

Contents
  paircorr_ref.c   plain FP64 loop over (t, i, j, s, t0, a): Eqs. 3-6, Algorithm 2
  checks.py        independent restatements used only to pin the loop oracle
                   (FFT lattice cross-correlation, separable NUDFT)
  dynamics.py      FP64 Landau-Lifshitz RK4 (Eq. 2), Metropolis / heat-bath
                   (Section 2.1) and the learned-proposal MLP (forward/backward)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paircorr_ref.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no FP contraction).  Idempotent."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32p, f32p, f64p, i64p = (ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64))
            lib.oracle_pair_corr.restype = ctypes.c_int
            lib.oracle_pair_corr.argtypes = [i64, i64, i64, i64, i64, i32p, f32p, ctypes.c_int,
                                             i32p, i32p, ctypes.c_int, f32p, ctypes.c_double, i64,
                                             i64, f64p, ctypes.c_int, i64, i64, f64p, f64p, f64p,
                                             f64p, f64p, f64p, f64p, i64p]
            lib.oracle_pair_corr_eq4.restype = ctypes.c_int
            lib.oracle_pair_corr_eq4.argtypes = [i64, i64, i64, i64, i64, i32p, f32p, ctypes.c_int,
                                                 i32p, i32p, ctypes.c_int, f32p, ctypes.c_double,
                                                 i64, f64p]
            lib.oracle_pair_counts.restype = ctypes.c_int
            lib.oracle_pair_counts.argtypes = [i64, ctypes.c_int, i32p, i32p, ctypes.c_int, f32p,
                                               ctypes.c_double, i64, i64, i64, i64p]
            lib.oracle_bin_of_d2.restype = ctypes.c_int
            lib.oracle_bin_of_d2.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_threads.argtypes = []
            lib.oracle_set_threads.restype = None
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_pair_d2.restype = ctypes.c_double
            lib.oracle_pair_d2.argtypes = [ctypes.c_int, i64, i64, i32p, i32p, ctypes.c_int, f32p]
            _lib = lib
    return _lib


def threads() -> int:
    """Threads the oracle's parallel loops use (for reporting a timing's core count)."""
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's following parallel loops."""
    _load().oracle_set_threads(int(n))


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


class Geometry:
    """Distance rule for the bins.  kind='lattice': integer coords + extents L,
    minimum image when periodic.  kind='positions': FP32 positions (FP32 rule)."""

    def __init__(self, kind, coords=None, L=(1, 1, 1), periodic=False, pos=None):
        assert kind in ("lattice", "positions")
        self.kind = kind
        self.coords = None if coords is None else np.ascontiguousarray(coords, np.int32)
        self.L = np.ascontiguousarray(L, np.int32)
        self.periodic = bool(periodic)
        self.pos = None if pos is None else np.ascontiguousarray(pos, np.float32)
        n = self.coords.shape[0] if self.coords is not None else self.pos.shape[0]
        if self.coords is None:
            self.coords = np.zeros((n, 3), np.int32)
        if self.pos is None:
            self.pos = self.coords.astype(np.float32)

    @property
    def geom(self):
        return 0 if self.kind == "lattice" else 1

    @classmethod
    def of_lattice(cls, lat, use_positions=None):
        if use_positions or (use_positions is None and not np.array_equal(lat.pos, lat.coords.astype(np.float32))):
            return cls("positions", coords=lat.coords, L=lat.L, periodic=False, pos=lat.pos)
        return cls("lattice", coords=lat.coords, L=lat.L, periodic=lat.periodic, pos=lat.pos)


def pair_corr(traj, T0, t_list, geometry: Geometry, w, n_bins, q=None, center=False,
              rows=None):
    """Binned sums and phase sums of Eqs. 3-6 (see paircorr_ref.c).

    traj [N][S][F][3] (or [N][F][3]) FP32.  Returns dict with C_sum, M_abs, P_abs
    [n_t][n_bins], Sq_sum (cosine part), Sq_im (sine part) and their magnitude sums
    Sq_abs, Sq_im_abs [n_t][n_q], counts [n_bins] (int64), all over the rows
    `rows=(i0,i1)` (default all) and every column."""
    lib = _load()
    tr = np.asarray(traj, np.float32)
    if tr.ndim == 3:
        tr = tr[:, None]
    tr = np.ascontiguousarray(tr)
    N, S, F, _ = tr.shape
    tl = np.ascontiguousarray(np.atleast_1d(t_list), np.int32)
    n_tl = tl.shape[0]
    qq = None if q is None or len(q) == 0 else np.ascontiguousarray(q, np.float64)
    n_q = 0 if qq is None else qq.shape[0]
    i0, i1 = (0, N) if rows is None else rows
    C = np.zeros((n_tl, n_bins))
    M = np.zeros((n_tl, n_bins))
    P = np.zeros((n_tl, n_bins))
    Sq = np.zeros((n_tl, max(n_q, 1)))
    Sqi = np.zeros((n_tl, max(n_q, 1)))
    Sqa = np.zeros((n_tl, max(n_q, 1)))
    Sqia = np.zeros((n_tl, max(n_q, 1)))
    cnt = np.zeros(n_bins, np.int64)
    g = geometry
    rc = lib.oracle_pair_corr(N, F, S, T0, n_tl, _p(tl, ctypes.c_int32), _p(tr, ctypes.c_float),
                              g.geom, _p(g.coords, ctypes.c_int32), _p(g.L, ctypes.c_int32),
                              int(g.periodic), _p(g.pos, ctypes.c_float), float(w), n_bins, n_q,
                              _p(qq, ctypes.c_double), int(bool(center)), i0, i1,
                              _p(C, ctypes.c_double), _p(M, ctypes.c_double),
                              _p(P, ctypes.c_double), _p(Sq, ctypes.c_double),
                              _p(Sqi, ctypes.c_double), _p(Sqa, ctypes.c_double),
                              _p(Sqia, ctypes.c_double), _p(cnt, ctypes.c_int64))
    if rc != 0:
        raise ValueError(f"oracle_pair_corr rejected its arguments (code {rc})")
    return {"C_sum": C, "M_abs": M, "P_abs": P, "Sq_sum": Sq[:, :n_q], "Sq_im": Sqi[:, :n_q],
            "Sq_abs": Sqa[:, :n_q], "Sq_im_abs": Sqia[:, :n_q], "counts": cnt,
            "N": N, "S": S, "T0": T0}


def pair_corr_eq4(traj, T0, t_list, geometry: Geometry, w, n_bins):
    """Eq. 4 form (product average minus product of averages), binned."""
    lib = _load()
    tr = np.asarray(traj, np.float32)
    if tr.ndim == 3:
        tr = tr[:, None]
    tr = np.ascontiguousarray(tr)
    N, S, F, _ = tr.shape
    tl = np.ascontiguousarray(np.atleast_1d(t_list), np.int32)
    C = np.zeros((tl.shape[0], n_bins))
    g = geometry
    lib.oracle_pair_corr_eq4(N, F, S, T0, tl.shape[0], _p(tl, ctypes.c_int32),
                             _p(tr, ctypes.c_float), g.geom, _p(g.coords, ctypes.c_int32),
                             _p(g.L, ctypes.c_int32), int(g.periodic), _p(g.pos, ctypes.c_float),
                             float(w), n_bins, _p(C, ctypes.c_double))
    return C


def pair_counts(geometry: Geometry, w, n_bins, rows=None):
    lib = _load()
    g = geometry
    N = g.coords.shape[0]
    i0, i1 = (0, N) if rows is None else rows
    cnt = np.zeros(n_bins, np.int64)
    lib.oracle_pair_counts(N, g.geom, _p(g.coords, ctypes.c_int32), _p(g.L, ctypes.c_int32),
                           int(g.periodic), _p(g.pos, ctypes.c_float), float(w), n_bins, i0, i1,
                           _p(cnt, ctypes.c_int64))
    return cnt


def bin_of_d2(d2, w):
    return _load().oracle_bin_of_d2(float(d2), float(w))


def pair_d2(geometry: Geometry, i, j):
    g = geometry
    return _load().oracle_pair_d2(g.geom, int(i), int(j), _p(g.coords, ctypes.c_int32),
                                  _p(g.L, ctypes.c_int32), int(g.periodic),
                                  _p(g.pos, ctypes.c_float))


def normalize(res):
    """C(b,t) = C_sum / (S*T0*n_b); S(q,t) = Sq_sum / (N*S*T0) (Eq. 3's 1/N)."""
    S, T0, N = res["S"], res["T0"], res["N"]
    n = res["counts"].astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        C = np.where(n > 0, res["C_sum"] / (S * T0 * np.maximum(n, 1)), 0.0)
    Sq = res["Sq_sum"] / (N * S * T0)
    return C, Sq


def rounding_ratio(C_sum_test, res):
    """|C_test - C_ref| / P_abs per bin: the error in units of the sum of absolute
    products, the quantity every rounding-error bound of the contraction scales with."""
    d = np.abs(np.asarray(C_sum_test, np.float64) - res["C_sum"])
    P = res["P_abs"]
    return np.where(P > 0, d / np.where(P > 0, P, 1.0), d)


def bin_error(C_sum_test, res):
    """Per-bin error of a tested C_sum against the oracle, scaled by the bin's
    magnitude sum: err_b(t) = |C_test - C_ref| / M_abs (both unnormalised, so the
    common 1/(S*T0*n_b) cancels).  Bins with M_abs == 0 use the absolute error."""
    ref, M = res["C_sum"], res["M_abs"]
    d = np.abs(np.asarray(C_sum_test, np.float64) - ref)
    return np.where(M > 0, d / np.where(M > 0, M, 1.0), d)


def sampled_bin_error(C_sum_test, res, min_pairs=16):
    """bin_error over the bins that hold at least `min_pairs` ordered pairs of the sample,
    0 elsewhere.  A row sample of a large problem leaves its far bins with a handful of
    pairs, where the per-bin error is the error of single pair terms; those bins are
    held to the rounding scale instead (rounding_ratio)."""
    e = bin_error(C_sum_test, res)
    return np.where(np.asarray(res["counts"])[None, :] >= min_pairs, e, 0.0)


def phase_error(Sq_test, res, part="cos"):
    """Per-(t, q) error of a tested phase sum against the oracle, scaled by that q's
    magnitude sum: |Sq_test - Sq_ref| / Sq_abs (cosine part) or against Sq_im with
    Sq_im_abs (sine part).  Entries with a zero scale use the absolute error."""
    ref, A = (res["Sq_sum"], res["Sq_abs"]) if part == "cos" else (res["Sq_im"], res["Sq_im_abs"])
    d = np.abs(np.asarray(Sq_test, np.float64) - ref)
    return np.where(A > 0, d / np.where(A > 0, A, 1.0), d)
