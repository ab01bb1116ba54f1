"""GPU parity of asd_pair_corr (all precision forms) against the FP64 oracle.

Tolerances (per-bin error scaled by the bin's magnitude sum, see oracle.bin_error; per-(t, q)
phase error scaled by that q's magnitude sum, see oracle.phase_error):
  FP32 and split-BF16: 1e-5 (the accuracy bar of the FP32-accurate forms);
  TF32: 4 * 2^-11 and BF16: 4 * 2^-8 (a few units of the operand rounding, the
  per-product error of a single rounded operand pair being <= 2u).
Pair counts are integers and must match exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 1e-5, "tf32": 4 * 2.0 ** -11, "bf16": 4 * 2.0 ** -8}
# Worst-case bound per unit of sum|A B| (first order): operand rounding of the form
# (split: the dropped lo*lo and residual terms, 3 * 2^-16; TF32 / BF16: two roundings,
# 2u) plus FP32 accumulation over K terms and the FP32 bin sums of one tile (a private
# bin of the tensor-core epilogue takes at most 256 adds; a per-warp bin copy of the
# FP32 form, 32 lanes x 64 pairs, at most 2048).
U32 = 2.0 ** -24


def elem_bound(form, K):
    per = {"fp32": 0.0, "split_bf16": 3 * 2.0 ** -16, "tf32": 2 * 2.0 ** -11,
           "bf16": 2 * 2.0 ** -8}[form]
    return per + (K + (2048 if form == "fp32" else 256)) * U32
FORMS = ["fp32", "split_bf16", "tf32", "bf16"]


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def run_gpu(asd, lat, traj, T0, n_t, w, n_bins, form, center=False, q=None, rows=None,
            tile_n=0, positions=None):
    tr = np.ascontiguousarray(traj if traj.ndim == 4 else traj[:, None])
    N, S, F, _ = tr.shape
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, n_bins, precision=form, S=S,
                                    center=center, q=q, positions=positions, tile_n=tile_n)
    d_tr = torch.from_numpy(tr).cuda()
    C = torch.zeros((n_t, max(n_bins, 1)), dtype=torch.float64, device="cuda")
    nq = 0 if q is None else len(q)
    Sq = torch.zeros((n_t, max(nq, 1)), dtype=torch.float64, device="cuda")
    plan.run(d_tr, C if n_bins else None, Sq if nq else None, rows=rows)
    assert asd.sync_status() == 0
    out = {"C_sum": C.cpu().numpy()[:, :n_bins], "Sq_sum": Sq.cpu().numpy()[:, :nq],
           "counts": plan.counts()}
    plan.close()
    return out


def oracle_ref(lat, traj, T0, n_t, w, n_bins, center=False, q=None, rows=None, positions=None):
    geo = oracle.Geometry.of_lattice(lat, use_positions=positions)
    return oracle.pair_corr(traj, T0, list(range(n_t)), geo, w, n_bins, q=q, center=center,
                            rows=rows)


def assert_parity(got, ref, form, q=False):
    err = oracle.bin_error(got["C_sum"], ref)
    assert err.max() <= TOL[form], f"{form}: max binned error {err.max():.3e}"
    if q:
        assert_phase(got["Sq_sum"], ref, form)


def assert_phase(sq, ref, form, part="cos"):
    """Every (t, q) of a phase sum within the form's tolerance of the oracle, in units of
    that q's magnitude sum."""
    d = oracle.phase_error(sq, ref, part)
    assert d.max() <= TOL[form], f"{form}: {part} phase error {d.max():.3e}"


@pytest.mark.parametrize("form", FORMS)
def test_square16_periodic(asd, form):
    """16x16 periodic square lattice (N=256, F=96, T0=64, 32 displacements, w=1)."""
    cfg = synth.cfg_small_2d()
    tr = synth.traj_precess(cfg.lattice.n_sites, cfg.F, seed=cfg.seed)
    got = run_gpu(asd, cfg.lattice, tr, cfg.T0, cfg.n_t, cfg.w, cfg.n_bins, form)
    ref = oracle_ref(cfg.lattice, tr, cfg.T0, cfg.n_t, cfg.w, cfg.n_bins)
    np.testing.assert_array_equal(got["counts"], ref["counts"])
    assert_parity(got, ref, form)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("center", [False, True])
def test_ragged_cubic_samples(asd, form, center):
    """7^3 = 343 sites (ragged against 128-row tiles), 2 samples, i.i.d. spins."""
    lat = synth.hypercubic(7, 3, True)
    tr = synth.traj_iid(lat.n_sites, 23, seed=17, S=2)
    got = run_gpu(asd, lat, tr, 13, 11, 0.5, 11, form, center=center)
    ref = oracle_ref(lat, tr, 13, 11, 0.5, 11, center=center)
    np.testing.assert_array_equal(got["counts"], ref["counts"])
    assert_parity(got, ref, form)


@pytest.mark.parametrize("form", FORMS)
def test_positions_with_phase(asd, form):
    """Jittered open cube (FP32 position rule) with cosine phase weights."""
    lat = synth.hypercubic(6, 3, False, jitter=0.1, seed=3)
    q = synth.q_vectors_glass()[::5]
    tr = synth.traj_precess(lat.n_sites, 40, seed=8)
    got = run_gpu(asd, lat, tr, 24, 9, 0.5, 20, form, q=q)
    ref = oracle_ref(lat, tr, 24, 9, 0.5, 20, q=q)
    np.testing.assert_array_equal(got["counts"], ref["counts"])
    assert_parity(got, ref, form, q=True)


@pytest.mark.parametrize("form", ["split_bf16", "bf16"])
def test_positions_two_windows(asd, form):
    """32^3 jittered glass in 4 x 4 x 8 site blocks, 256 bins of 0.5, of which the private
    window holds 81 (8 epilogue warps).  A 192-column tile that joins the last sites of one
    row of blocks with the first sites of the next spans more bins than that, and is
    binned through two windows, one per group of its 32-column chunks; each of the first
    two row tiles meets one such tile.  Bins and 16 q-vectors against the oracle."""
    lat = synth.hypercubic(32, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 8),
                           jitter=0.1)
    q = synth.q_vectors_glass()[::4]
    tr = synth.traj_precess(lat.n_sites, 34, seed=9)
    rows = (0, 256)
    got = run_gpu(asd, lat, tr, 32, 2, 0.5, 256, form, q=q, rows=rows)
    ref = oracle_ref(lat, tr, 32, 2, 0.5, 256, q=q, rows=rows)
    assert_parity(got, ref, form, q=True)


@pytest.mark.parametrize("form", ["split_bf16", "fp32"])
def test_row_range(asd, form):
    lat = synth.hypercubic(20, 2, True)
    tr = synth.traj_precess(lat.n_sites, 30, seed=5)
    rows = (37, 301)
    got = run_gpu(asd, lat, tr, 16, 8, 1.0, 15, form, rows=rows)
    ref = oracle_ref(lat, tr, 16, 8, 1.0, 15, rows=rows)
    assert_parity(got, ref, form)


@pytest.mark.parametrize("form", FORMS)
def test_window_bins(asd, form):
    """Many narrow bins (a few pairs each, so no averaging): private-bin window plus the
    shared fallback path; error held to the per-element rounding bound."""
    lat = synth.hypercubic(8, 3, False, jitter=0.1, seed=4, block=(4, 4, 2))
    tr = synth.traj_precess(lat.n_sites, 20, seed=6)
    got = run_gpu(asd, lat, tr, 12, 5, 0.01, 1500, form)
    ref = oracle_ref(lat, tr, 12, 5, 0.01, 1500)
    np.testing.assert_array_equal(got["counts"], ref["counts"])
    r = oracle.rounding_ratio(got["C_sum"], ref)
    assert r.max() <= elem_bound(form, 36), f"{form}: {r.max():.3e}"


@pytest.mark.parametrize("form", FORMS)
def test_degenerate_single_site(asd, form):
    lat = synth.hypercubic(1, 2, True)
    tr = synth.traj_iid(1, 5, seed=2)
    got = run_gpu(asd, lat, tr, 5, 1, 1.0, 1, form)
    ref = oracle_ref(lat, tr, 5, 1, 1.0, 1)
    assert got["counts"][0] == 1
    assert_parity(got, ref, form)


@pytest.mark.parametrize("form", ["split_bf16", "tf32"])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_tile_widths_static_fm(asd, form, tile_n):
    """Static ferromagnet: C == 1 in every bin, for both tile widths."""
    lat = synth.hypercubic(9, 3, True)
    tr = synth.traj_static(lat.n_sites, 12, direction=(0.3, -0.4, 0.866))
    got = run_gpu(asd, lat, tr, 8, 4, 0.5, 13, form, tile_n=tile_n)
    n = got["counts"].astype(np.float64)
    full = n > 0                       # w = 0.5 leaves bins without lattice pairs
    assert full.sum() >= 8
    C = got["C_sum"][:, full] / (8 * n[full])
    # identical products do not average: the worst-case per-product bound applies
    np.testing.assert_allclose(C, 1.0, rtol=0, atol=elem_bound(form, 24))


@pytest.mark.parametrize("form", ["split_bf16", "bf16", "tf32"])
@pytest.mark.parametrize("k_chunks", [1, 3, 4])
def test_k_chunks(asd, form, k_chunks):
    """K split into partial accumulators (9^3 = 729 sites: 6 row tiles, the last ragged),
    over all rows and over a row range that starts mid-tile."""
    lat = synth.hypercubic(9, 3, True)
    tr = synth.traj_precess(lat.n_sites, 70, seed=21, S=2)
    for rows in (None, (100, 700)):
        tr2 = np.ascontiguousarray(tr)
        N, S, F, _ = tr2.shape
        plan = asd.CorrPlan.for_lattice(lat, F, 40, 6, 0.5, 14, precision=form, S=S,
                                        k_chunks=k_chunks)
        d_tr = torch.from_numpy(tr2).cuda()
        C = torch.zeros((6, 14), dtype=torch.float64, device="cuda")
        plan.run(d_tr, C, rows=rows)
        assert asd.sync_status() == 0
        ref = oracle_ref(lat, tr, 40, 6, 0.5, 14, rows=rows)
        assert_parity({"C_sum": C.cpu().numpy()}, ref, form)
        plan.close()


# lattice binning variants: packed-coordinate d2 with the d2 -> bin table (periodic and
# open), packed d2 with thresholds (table too large), the general path (coordinates past
# one byte), and too few bins (dropped pairs go to the trash row)
LATTICE_CASES = {
    "periodic_table_dropped": (lambda: synth.hypercubic(12, 3, True), 0.5, 9, None),
    "open_table": (lambda: synth.hypercubic(11, 3, False), 1.0, 12, None),
    "periodic_thresholds": (lambda: synth.hypercubic(190, 2, True), 1.0, 60, (1000, 1100)),
    "open_wide_general": (lambda: synth.hypercubic(130, 2, False), 2.0, 50, (16000, 16100)),
    "periodic_256_general": (lambda: synth.hypercubic(256, 2, True), 1.5, 70, (30000, 30100)),
}


@pytest.mark.parametrize("form", ["split_bf16", "bf16"])
@pytest.mark.parametrize("case", sorted(LATTICE_CASES))
def test_lattice_binning_paths(asd, form, case):
    make, w, nb, rows = LATTICE_CASES[case]
    lat = make()
    tr = synth.traj_precess(lat.n_sites, 14, seed=31)
    got = run_gpu(asd, lat, tr, 8, 5, w, nb, form, rows=rows)
    ref = oracle_ref(lat, tr, 8, 5, w, nb, rows=rows)
    if rows is None:
        np.testing.assert_array_equal(got["counts"], ref["counts"])
    assert_parity(got, ref, form)


@pytest.mark.parametrize("form", ["split_bf16", "bf16", "tf32"])
def test_phase_on_lattice_row_range(asd, form):
    """Phase weights on integer lattice coordinates (square-lattice q path, 21 q: a
    partial last pass), bins at the same time, rows starting and ending mid-tile."""
    lat = synth.hypercubic(20, 2, True)
    q = synth.q_path_square(20)[:21]
    tr = synth.traj_precess(lat.n_sites, 30, seed=12)
    rows = (37, 301)
    got = run_gpu(asd, lat, tr, 16, 6, 1.0, 15, form, q=q, rows=rows)
    ref = oracle_ref(lat, tr, 16, 6, 1.0, 15, q=q, rows=rows)
    assert_parity(got, ref, form, q=True)


@pytest.mark.parametrize("form", ["split_bf16", "bf16", "tf32"])
@pytest.mark.parametrize("tile_n,ew", [(128, 4), (192, 4), (192, 8)])
@pytest.mark.parametrize("sine", [False, True])
def test_phase_tile_widths(asd, form, tile_n, ew, sine):
    """The tensor-core phase product at both tile widths that leave it TMEM room, with 4
    and 8 epilogue warps: 13 q (a partial pass), bins at the same time, rows from mid-tile
    (ragged row and column tiles), cosine and sine parts.  Wider tiles are refused."""
    lat = synth.hypercubic(9, 3, False, jitter=0.1, seed=5)
    q = synth.q_vectors_glass()[::5]
    tr = synth.traj_precess(lat.n_sites, 30, seed=9)
    rows = (20, 700)
    plan = asd.CorrPlan.for_lattice(lat, 30, 18, 7, 0.5, 16, precision=form, q=q,
                                    phase_sine=sine, tile_n=tile_n, epi_warps=ew)
    C = torch.zeros((7, 16), dtype=torch.float64, device="cuda")
    Sq = torch.zeros((7, len(q), 2) if sine else (7, len(q)), dtype=torch.float64,
                     device="cuda")
    plan.run(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda(), C, Sq, rows=rows)
    assert asd.sync_status() == 0
    plan.close()
    ref = oracle.pair_corr(tr, 18, list(range(7)), oracle.Geometry.of_lattice(lat), 0.5, 16,
                           q=q, rows=rows)
    got = Sq.cpu().numpy()
    assert_phase(got[..., 0] if sine else got, ref, form)
    if sine:
        assert_phase(got[..., 1], ref, form, "sin")
    assert oracle.bin_error(C.cpu().numpy(), ref).max() <= TOL[form]
    for kw in ({"tile_n": 256}, {"tile_n": 128, "epi_warps": 8}):
        with pytest.raises(asd.AsdError):
            asd.CorrPlan.for_lattice(lat, 30, 18, 7, 0.5, 16, precision=form, q=q, **kw)


@pytest.mark.parametrize("form", FORMS)
def test_phase_sine_part(asd, form):
    """Cosine and sine parts of Eq. 3's phase sum (jittered open cube, 13 q, rows from
    mid-tile), in the [n_t][n_q][2] layout; the sine part vanishes at t = 0."""
    lat = synth.hypercubic(7, 3, False, jitter=0.1, seed=3)
    q = synth.q_vectors_glass()[::5]
    tr = synth.traj_precess(lat.n_sites, 30, seed=8)
    rows = (20, 300)
    plan = asd.CorrPlan.for_lattice(lat, 30, 18, 9, 0.5, 12, precision=form, q=q,
                                    phase_sine=True)
    C = torch.zeros((9, 12), dtype=torch.float64, device="cuda")
    Sq = torch.zeros((9, len(q), 2), dtype=torch.float64, device="cuda")
    plan.run(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda(), C, Sq, rows=rows)
    Sep = torch.zeros((9, len(q), 2), dtype=torch.float64, device="cuda")
    plan.sq_separable(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda(), Sep)
    assert asd.sync_status() == 0
    plan.close()
    ref = oracle.pair_corr(tr, 18, list(range(9)), oracle.Geometry.of_lattice(lat), 0.5, 12,
                           q=q, rows=rows)
    full = oracle.pair_corr(tr, 18, list(range(9)), oracle.Geometry.of_lattice(lat), 0.5, 1, q=q)
    got = Sq.cpu().numpy()
    assert_phase(got[..., 0], ref, form)
    assert_phase(got[..., 1], ref, form, "sin")
    assert oracle.bin_error(C.cpu().numpy(), ref).max() <= TOL[form]
    sep = Sep.cpu().numpy()
    assert_phase(sep[..., 0], full, "fp32")
    assert_phase(sep[..., 1], full, "fp32", "sin")
    assert np.abs(sep[0, :, 1]).max() <= 1e-5 * full["Sq_im_abs"][0].max()


@pytest.mark.parametrize("form", FORMS)
def test_rows_past_the_range_are_ignored(asd, form):
    """A rows outside the contracted range may hold anything (here NaN from an earlier
    preparation of the whole range): bins, phase and sine parts of the range stay
    exact.  Positions geometry (threshold binning) with phase weights."""
    lat = synth.hypercubic(7, 3, False, jitter=0.1, seed=3)
    q = synth.q_vectors_glass()[::5]
    tr = synth.traj_precess(lat.n_sites, 30, seed=8)
    bad = np.full_like(tr, np.nan)
    rows = (20, 300)
    plan = asd.CorrPlan.for_lattice(lat, 30, 18, 9, 0.5, 12, precision=form, q=q,
                                    phase_sine=True)
    plan.prepare(torch.from_numpy(np.ascontiguousarray(bad[:, None])).cuda())
    d_tr = torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda()
    plan.prepare(d_tr, rows=rows)
    C = torch.zeros((9, 12), dtype=torch.float64, device="cuda")
    Sq = torch.zeros((9, len(q), 2), dtype=torch.float64, device="cuda")
    plan.contract(C, Sq, rows=rows)
    assert asd.sync_status() == 0
    plan.close()
    got_c, got_q = C.cpu().numpy(), Sq.cpu().numpy()
    assert np.isfinite(got_c).all() and np.isfinite(got_q).all()
    ref = oracle.pair_corr(tr, 18, list(range(9)), oracle.Geometry.of_lattice(lat), 0.5, 12,
                           q=q, rows=rows)
    assert oracle.bin_error(got_c, ref).max() <= TOL[form]
    assert_phase(got_q[..., 0], ref, form)
    assert_phase(got_q[..., 1], ref, form, "sin")


@pytest.mark.parametrize("form", ["split_bf16", "bf16", "tf32", "fp32"])
def test_degenerate_shapes(asd, form):
    """The paper's own averaging (one origin, M samples: T0 = 1, S = M), one displacement
    with F = T0 + n_t - 1 exactly, a single bin, and an empty row range (a no-op)."""
    lat = synth.hypercubic(9, 2, True)
    # M = 50 realisations at one origin, 3 frames: K = 3 * 1 * 50
    tr = synth.traj_precess(lat.n_sites, 3, seed=14, S=50)
    got = run_gpu(asd, lat, tr, 1, 3, 1.0, 7, form)
    ref = oracle_ref(lat, tr, 1, 3, 1.0, 7)
    assert_parity(got, ref, form)
    # a single displacement, F = T0 exactly, one bin (every pair within r < w)
    tr2 = synth.traj_precess(lat.n_sites, 16, seed=15)
    got = run_gpu(asd, lat, tr2, 16, 1, 100.0, 1, form)
    ref = oracle_ref(lat, tr2, 16, 1, 100.0, 1)
    assert got["counts"][0] == lat.n_sites ** 2
    assert_parity(got, ref, form)
    # empty row range: nothing is added
    got = run_gpu(asd, lat, tr2, 8, 4, 1.0, 7, form, rows=(40, 40))
    assert not got["C_sum"].any()


def test_maximum_q_count(asd):
    """n_q = 256 (the largest accepted): all phase passes, every chunk full."""
    lat = synth.hypercubic(5, 3, False, jitter=0.1, seed=2)
    g = np.random.default_rng(3)
    q = g.standard_normal((256, 3))
    tr = synth.traj_precess(lat.n_sites, 12, seed=6)
    got = run_gpu(asd, lat, tr, 8, 3, 0.5, 6, "split_bf16", q=q)
    ref = oracle_ref(lat, tr, 8, 3, 0.5, 6, q=q)
    assert_parity(got, ref, "split_bf16", q=True)


@pytest.mark.parametrize("form", ["split_bf16", "fp32", "bf16"])
def test_displacement_range(asd, form):
    """asd_pair_corr_contract_range: displacements in blocks [0, 3), [3, 7), [7, 11)
    accumulate into one output (bins and phase, rows from mid-tile) and match the oracle;
    a single block touches only its own rows of the outputs; an empty or reversed range
    is a no-op or an error."""
    lat = synth.hypercubic(7, 3, False, jitter=0.1, seed=3)
    q = synth.q_vectors_glass()[::5]
    tr = synth.traj_precess(lat.n_sites, 30, seed=8)
    rows = (20, 300)
    plan = asd.CorrPlan.for_lattice(lat, 30, 18, 11, 0.5, 12, precision=form, q=q)
    plan.prepare(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda())
    C = torch.zeros((11, 12), dtype=torch.float64, device="cuda")
    Sq = torch.zeros((11, len(q)), dtype=torch.float64, device="cuda")
    for tb in ((0, 3), (3, 7), (7, 11), (5, 5)):
        plan.contract(C, Sq, rows=rows, t_range=tb)
    C1 = torch.zeros_like(C)
    plan.contract(C1, torch.zeros_like(Sq), rows=rows, t_range=(3, 7))
    with pytest.raises(asd.AsdError):
        plan.contract(C1, torch.zeros_like(Sq), rows=rows, t_range=(7, 3))
    with pytest.raises(asd.AsdError):
        plan.contract(C1, torch.zeros_like(Sq), rows=rows, t_range=(0, 12))
    assert asd.sync_status() == 0
    plan.close()
    ref = oracle.pair_corr(tr, 18, list(range(11)), oracle.Geometry.of_lattice(lat), 0.5, 12,
                           q=q, rows=rows)
    assert_parity({"C_sum": C.cpu().numpy(), "Sq_sum": Sq.cpu().numpy()}, ref, form, q=True)
    c1 = C1.cpu().numpy()
    assert not c1[:3].any() and not c1[7:].any() and c1[3:7].any()
    assert oracle.bin_error(c1[3:7], {k: (v[3:7] if k in ("C_sum", "M_abs") else v)
                                      for k, v in ref.items()}).max() <= TOL[form]
