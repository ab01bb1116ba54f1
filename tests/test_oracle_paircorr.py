"""Pins of the FP64 pair-correlation oracle against values fixed by the paper and by
mathematics (hand-computed cases, closed forms, invariants, independent algorithms).
None of these re-types the oracle's own loop."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import checks
from paper_2308_07487_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _two_site_geom():
    coords = np.array([[0, 0, 0], [1, 0, 0]], np.int32)
    return oracle.Geometry("lattice", coords=coords, L=(2, 1, 1), periodic=False)


def test_two_site_hand_computed():
    g = _load("two_site_hand.json")
    traj = np.array(g["traj"], np.float32)
    geo = _two_site_geom()
    r = oracle.pair_corr(traj, g["T0"], g["t_list"], geo, g["w"], g["n_bins"], q=np.array(g["q"]))
    np.testing.assert_allclose(r["C_sum"], g["C_sum"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["M_abs"], g["M_abs"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["counts"], g["counts"])
    np.testing.assert_allclose(r["Sq_sum"], g["Sq_sum"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["P_abs"], g["P_abs"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Sq_abs"], g["Sq_abs"], rtol=0, atol=1e-12)
    rc = oracle.pair_corr(traj, g["T0"], g["t_list"], geo, g["w"], g["n_bins"], center=True,
                          q=np.array(g["q"]))
    np.testing.assert_allclose(rc["C_sum"], g["C_sum_center"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(rc["M_abs"], g["M_abs_center"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(rc["P_abs"], g["P_abs_center"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(rc["Sq_sum"], g["Sq_sum_center"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(rc["Sq_abs"], g["Sq_abs_center"], rtol=0, atol=1e-12)


def test_two_site_mixed_signs_hand_computed():
    """Scales of the error metrics: M_abs = sum|G| (not |sum G|), P_abs = sum|A B| (not
    sum|G|), Sq_abs = sum|cos G| per q and the sine part with its scale, on a case where
    each of those differs from the quantity it could be mistaken for."""
    g = _load("two_site_signs.json")
    traj = np.array(g["traj"], np.float32)
    r = oracle.pair_corr(traj, g["T0"], g["t_list"], _two_site_geom(), g["w"], g["n_bins"],
                         q=np.array(g["q"]))
    for k in ("C_sum", "M_abs", "P_abs", "Sq_sum", "Sq_abs", "Sq_im", "Sq_im_abs"):
        np.testing.assert_allclose(r[k], g[k], rtol=0, atol=1e-12, err_msg=k)
    np.testing.assert_array_equal(r["counts"], g["counts"])
    # the error helpers divide by exactly these scales
    bumped = r["C_sum"] + 0.3
    np.testing.assert_allclose(oracle.bin_error(bumped, r)[1], 0.3 / np.array(g["M_abs"][1]))
    np.testing.assert_allclose(oracle.rounding_ratio(bumped, r)[1], 0.3 / np.array(g["P_abs"][1]))
    np.testing.assert_allclose(oracle.phase_error(r["Sq_sum"] + 0.7, r)[1],
                               0.7 / np.array(g["Sq_abs"][1]))
    np.testing.assert_allclose(oracle.phase_error(r["Sq_im"] + 0.2, r, "sin")[1, 0], 0.2 / 4)
    # the sampled per-bin error keeps bins with enough pairs and zeroes the others
    np.testing.assert_array_equal(oracle.sampled_bin_error(bumped, r, min_pairs=2),
                                  oracle.bin_error(bumped, r))
    assert not oracle.sampled_bin_error(bumped, r, min_pairs=3).any()


def test_bin_rule_golden():
    g = _load("bin_rule.json")
    for c in g["cases"]:
        assert oracle.bin_of_d2(c["d2"], c["w"]) == c["bin"], c


def test_square_lattice_shell_counts():
    g = _load("bin_rule.json")
    lat = synth.hypercubic(16, 2, True)
    geo = oracle.Geometry.of_lattice(lat)
    cnt = oracle.pair_counts(geo, 1.0, 12)
    assert list(cnt[:3]) == g["sq16_w1_counts_first3"]
    assert cnt.sum() == 256 * 256          # every ordered pair lands in one of the 12 bins
    # shells from the textbook table: number of displacement vectors with each |d|^2
    shells = {int(k): v for k, v in g["square_shells"].items()}
    assert cnt[0] == 256 * shells[0]
    assert cnt[1] == 256 * (shells[1] + shells[2])
    assert cnt[2] == 256 * (shells[4] + shells[5] + shells[8])


def _isqrt_bin_counts(L, dim, w2x):
    """Independent count: bin = isqrt(d2 * w2x) for w = 1/sqrt(w2x) with w2x in {1,4}."""
    Ls = [L] * dim
    out = {}
    for d in itertools.product(*[range(v) for v in Ls]):
        d2 = sum(min(x, v - x) ** 2 for x, v in zip(d, Ls))
        b = math.isqrt(d2 * w2x)
        out[b] = out.get(b, 0) + 1
    return out


@pytest.mark.parametrize("L,dim,w", [(16, 2, 1.0), (6, 3, 0.5), (7, 2, 0.5)])
def test_lattice_counts_vs_integer_enumeration(L, dim, w):
    lat = synth.hypercubic(L, dim, True)
    geo = oracle.Geometry.of_lattice(lat)
    ref = _isqrt_bin_counts(L, dim, 1 if w == 1.0 else 4)
    n_bins = max(ref) + 1
    cnt = oracle.pair_counts(geo, w, n_bins)
    N = lat.n_sites
    for b in range(n_bins):
        assert cnt[b] == N * ref.get(b, 0)


def test_unit_spins_self_bin_is_one():
    """C(0, t=0) = 1 for unit spins: bin 0 holds exactly the self pairs on a lattice."""
    lat = synth.hypercubic(6, 3, True)
    geo = oracle.Geometry.of_lattice(lat)
    tr = synth.traj_iid(lat.n_sites, 20, seed=5)
    r = oracle.pair_corr(tr, 12, [0, 3], geo, 0.5, 8)
    C, _ = oracle.normalize(r)
    # FP32 unit vectors have |S|^2 = 1 within a few units of 2^-24
    assert abs(C[0, 0] - 1.0) < 4 * 2.0 ** -24
    assert abs(C[1, 0]) < 0.2               # decorrelated i.i.d. frames at t=3


def test_static_ferromagnet_is_one_everywhere():
    """C(b,t) = 1 for every bin and displacement in a static ferromagnetic state."""
    lat = synth.hypercubic(5, 2, True)
    geo = oracle.Geometry.of_lattice(lat)
    tr = synth.traj_static(lat.n_sites, 9, direction=(0.2, -0.5, 0.84), S=2)
    r = oracle.pair_corr(tr, 5, [0, 1, 4], geo, 1.0, 3)   # 5x5 periodic: d2 <= 8, bins 0..2
    assert (r["counts"] > 0).all()
    C, _ = oracle.normalize(r)
    np.testing.assert_allclose(C, 1.0, rtol=0, atol=4 * 2.0 ** -24)


@pytest.mark.parametrize("L,dim,periodic,w", [(8, 2, True, 1.0), (5, 3, True, 0.5),
                                              (6, 2, False, 1.0), (4, 3, False, 0.5)])
def test_fft_cross_correlation_matches(L, dim, periodic, w):
    """The lattice FFT route (an independent algorithm) gives the same binned sums."""
    lat = synth.hypercubic(L, dim, periodic)
    geo = oracle.Geometry.of_lattice(lat)
    S, F, T0 = 2, 17, 9
    tr = synth.traj_precess(lat.n_sites, F, seed=11, S=S)
    t_list = [0, 1, 5, 8]
    n_bins = int(math.isqrt(int(dim * (L if not periodic else L // 2) ** 2 / w ** 2))) + 1
    r = oracle.pair_corr(tr, T0, t_list, geo, w, n_bins)
    ref = checks.lattice_fft_corr(tr, T0, t_list, lat.coords, lat.L, periodic, w, n_bins)
    scale = np.abs(r["M_abs"]).max()
    np.testing.assert_allclose(r["C_sum"], ref, rtol=0, atol=1e-10 * scale)


def test_fft_check_on_block_numbered_sites():
    """Relabelling the sites (spatial blocks) leaves the binned sums unchanged."""
    lat_a = synth.hypercubic(8, 3, True)
    lat_b = synth.hypercubic(8, 3, True, block=(4, 4, 2))
    tr_a = synth.traj_iid(lat_a.n_sites, 10, seed=3)
    # same physical trajectory, rows permuted to the block numbering
    idx_a = {tuple(c): k for k, c in enumerate(lat_a.coords)}
    perm = np.array([idx_a[tuple(c)] for c in lat_b.coords])
    tr_b = tr_a[perm]
    ra = oracle.pair_corr(tr_a, 6, [0, 2], oracle.Geometry.of_lattice(lat_a), 0.5, 14)
    rb = oracle.pair_corr(tr_b, 6, [0, 2], oracle.Geometry.of_lattice(lat_b), 0.5, 14)
    np.testing.assert_allclose(ra["C_sum"], rb["C_sum"], rtol=1e-12, atol=1e-9)
    np.testing.assert_array_equal(ra["counts"], rb["counts"])


def test_phase_form_matches_separable_transform():
    """Phase-weighted sum (Eq. 3 with Eq. 6) equals the factorised NUDFT form."""
    lat = synth.hypercubic(4, 3, False, jitter=0.1, seed=7)
    geo = oracle.Geometry.of_lattice(lat)
    assert geo.kind == "positions"
    tr = synth.traj_precess(lat.n_sites, 14, seed=2)
    q = synth.q_vectors_glass()[::7]
    for center in (False, True):
        r = oracle.pair_corr(tr, 8, [0, 2, 6], geo, 0.5, 10, q=q, center=center)
        ref = checks.separable_phase_sum(tr, 8, [0, 2, 6], lat.pos, q, center=center)
        np.testing.assert_allclose(r["Sq_sum"], ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        ref_s = checks.separable_phase_sum(tr, 8, [0, 2, 6], lat.pos, q, center=center,
                                           part="sin")
        np.testing.assert_allclose(r["Sq_im"], ref_s, rtol=0, atol=1e-10 * np.abs(ref).max())
        # sine weights are odd and G(0) is symmetric: the sine part vanishes at t = 0
        assert np.abs(r["Sq_im"][0]).max() <= 1e-12 * np.abs(r["Sq_sum"]).max()
        assert np.abs(r["Sq_im"][1:]).max() > 1e-6 * np.abs(r["Sq_sum"]).max()


def test_q_zero_is_total_moment_correlation():
    lat = synth.hypercubic(5, 2, True)
    geo = oracle.Geometry.of_lattice(lat)
    tr = synth.traj_precess(lat.n_sites, 12, seed=4, S=3)
    r = oracle.pair_corr(tr, 6, [0, 3, 6], geo, 1.0, 5, q=np.zeros((1, 3)))
    ref = checks.total_moment_corr(tr, 6, [0, 3, 6])
    np.testing.assert_allclose(r["Sq_sum"][:, 0], ref, rtol=1e-12)


def test_eq4_equals_eq5():
    """Eq. 4 (mean product subtracted) and Eq. 5 (centred product) agree (Section 3.2)."""
    lat = synth.hypercubic(4, 2, True)
    geo = oracle.Geometry.of_lattice(lat)
    tr = synth.traj_precess(lat.n_sites, 11, seed=9, S=2)
    c5 = oracle.pair_corr(tr, 6, [0, 2, 5], geo, 1.0, 4, center=True)["C_sum"]
    c4 = oracle.pair_corr_eq4(tr, 6, [0, 2, 5], geo, 1.0, 4)
    np.testing.assert_allclose(c5, c4, rtol=1e-10, atol=1e-10)


def test_row_ranges_add_up():
    lat = synth.hypercubic(6, 2, True)
    geo = oracle.Geometry.of_lattice(lat)
    tr = synth.traj_iid(lat.n_sites, 8, seed=1)
    full = oracle.pair_corr(tr, 4, [0, 2], geo, 1.0, 6)
    parts = [oracle.pair_corr(tr, 4, [0, 2], geo, 1.0, 6, rows=(a, b))
             for a, b in ((0, 7), (7, 20), (20, 36))]
    np.testing.assert_allclose(sum(p["C_sum"] for p in parts), full["C_sum"], atol=1e-12)
    assert (sum(p["counts"] for p in parts) == full["counts"]).all()


def test_position_rule_threshold_cases():
    """FP32 position rule at exact thresholds: d2 = 0.25 is bin 1 at w = 0.5."""
    pos = np.array([[0, 0, 0], [0.5, 0, 0], [np.nextafter(np.float32(0.5), np.float32(0)), 0, 0],
                    [0.3, 0.4, 0]], np.float32)
    geo = oracle.Geometry("positions", pos=pos)
    assert oracle.pair_d2(geo, 0, 1) == 0.25
    assert oracle.bin_of_d2(oracle.pair_d2(geo, 0, 1), 0.5) == 1
    assert oracle.bin_of_d2(oracle.pair_d2(geo, 0, 2), 0.5) == 0
    # 0.3^2 + 0.4^2 in FP32 with one fma: close to 0.25 -> compare with an explicit float32 eval
    dx, dy = np.float32(0.3), np.float32(0.4)
    d2 = np.float32(np.float64(dy) * np.float64(dy) + np.float64(np.float32(dx * dx)))
    assert oracle.pair_d2(geo, 0, 3) == float(d2)


@pytest.mark.parametrize("periodic,jitter", [(True, 0.0), (False, 0.1)])
def test_time_reversal_swaps_the_pair_roles(periodic, jitter):
    """i <-> j symmetry: with F = T0 + n_t - 1 frames, reversing the trajectory in time
    maps displacement t_max = n_t - 1 onto itself with S_i(t0 + t) . S_j(t0) turned into
    S_j(u + t) . S_i(u) over the same origins; the bins and the phase weights are
    symmetric in (i, j) (cos is even), so the binned and phase sums at t_max are unchanged,
    while the other displacements move to other origin windows."""
    lat = synth.hypercubic(4, 3, periodic, jitter=jitter, seed=7)
    geo = oracle.Geometry.of_lattice(lat)
    T0, n_t = 6, 5
    F = T0 + n_t - 1
    tr = synth.traj_precess(lat.n_sites, F, seed=13, S=2)
    rev = np.ascontiguousarray(tr[:, :, ::-1])
    q = synth.q_vectors_glass()[::9]
    a = oracle.pair_corr(tr, T0, [n_t - 1], geo, 0.5, 8, q=q)
    b = oracle.pair_corr(rev, T0, [n_t - 1], geo, 0.5, 8, q=q)
    np.testing.assert_allclose(a["C_sum"], b["C_sum"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a["Sq_sum"], b["Sq_sum"], rtol=1e-12, atol=1e-12)
    # the sine weight is odd in (i, j): reversal flips the sign of the sine part
    np.testing.assert_allclose(a["Sq_im"], -b["Sq_im"], rtol=1e-12, atol=1e-12)
    # a planted swap of i and j in one term would break it: t = 1 is not invariant
    c = oracle.pair_corr(tr, T0, [1], geo, 0.5, 8)
    d = oracle.pair_corr(rev, T0, [1], geo, 0.5, 8)
    assert np.abs(c["C_sum"] - d["C_sum"]).max() > 1e-3
