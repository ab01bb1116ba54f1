"""Deterministic mode (asd_corr_desc.deterministic): every sum across threads, tiles and
CTAs in 64-bit fixed point, so C_sum / Sq_sum come out bit for bit the same for any work
schedule (dynamic or static order, raster height, stage count, order of a batch) and on
every repeat, while staying within the parity bar of the oracle.  Covered paths: the
branch-free lattice table path, the position path with a private window and the shared
fallback bins, the tensor-core phase product (cosine and sine parts), K-chunked split-BF16,
the FP32 form and the batched launch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def run(asd, lat, tr, T0, n_t, w, nb, form, q=None, sine=False, rows=None, **knobs):
    F = tr.shape[-2]  # trajectories are [N][S][F][3]
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision=form, q=q,
                                    phase_sine=sine, **knobs)
    d_tr = torch.from_numpy(np.ascontiguousarray(tr)).cuda()
    C = torch.zeros((n_t, max(nb, 1)), dtype=torch.float64, device="cuda")
    nq = 0 if q is None else len(q)
    Sq = torch.zeros((n_t, max(nq, 1), 1 + int(sine)), dtype=torch.float64, device="cuda")
    plan.run(d_tr, C if nb else None, Sq if nq else None, rows=rows)
    assert asd.sync_status() == 0
    plan.close()
    return C.cpu().numpy(), Sq.cpu().numpy()


def bits_equal(a, b):
    return np.array_equal(a.view(np.int64), b.view(np.int64))


# (lattice, T0, n_t, w, n_bins, q, sine, rows, forms, knob variants)
GLASS = lambda: synth.hypercubic(12, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 4),
                                 jitter=0.1)
CASES = {
    # positions, bins + phase (both parts), 2 K-chunks, rows from mid-tile
    "glass_phase": (GLASS, 96, 6, 0.5, 40, synth.q_vectors_glass()[::4], True, (37, 1700),
                    ["split_bf16", "bf16"], dict(k_chunks=2)),
    # positions, many narrow bins: private window + fallback bins
    "window_fallback": (lambda: synth.hypercubic(8, 3, False, jitter=0.1, seed=4, block=(4, 4, 2)),
                        12, 5, 0.01, 1500, None, False, None, ["split_bf16", "tf32"], {}),
    # periodic lattice, branch-free packed-coordinate table path
    "lattice_lut": (lambda: synth.hypercubic(14, 3, True), 24, 6, 0.5, 20, None, False, None,
                    ["split_bf16", "fp32"], {}),
}
SCHEDULES = [dict(), dict(static_schedule=True), dict(raster_m=3, stages=2)]


@pytest.mark.parametrize("case", sorted(CASES))
def test_bitwise_over_schedules(asd, case):
    make, T0, n_t, w, nb, q, sine, rows, forms, knobs = CASES[case]
    lat = make()
    F = T0 + n_t + 2
    tr = synth.traj_precess(lat.n_sites, F, seed=41)
    ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb,
                           q=q, rows=rows)
    for form in forms:
        scheds = SCHEDULES if form != "fp32" else [dict(), dict()]
        outs = [run(asd, lat, tr, T0, n_t, w, nb, form, q=q, sine=sine, rows=rows,
                    deterministic=True, **knobs, **sk) for sk in scheds]
        outs.append(run(asd, lat, tr, T0, n_t, w, nb, form, q=q, sine=sine, rows=rows,
                        deterministic=True, **knobs))  # a repeat of the first
        C0, S0 = outs[0]
        for C, S in outs[1:]:
            assert bits_equal(C, C0), f"{case} {form}: bins differ between schedules"
            assert bits_equal(S, S0), f"{case} {form}: phase sums differ between schedules"
        # the same sums as the default (floating-point atomics) mode to well below the bar:
        # the default mode's fallback bins are FP32 shared-memory sums (a few 2^-24 of
        # their magnitude), the fixed-point sums are exact to 2^-e
        Cf, Sf = run(asd, lat, tr, T0, n_t, w, nb, form, q=q, sine=sine, rows=rows, **knobs)
        m = ref["M_abs"] > 0
        assert (np.abs(C0[:, :nb] - Cf[:, :nb])[m] / ref["M_abs"][m]).max(initial=0) <= 1e-6
        tol = {"split_bf16": 1e-5, "fp32": 1e-5, "tf32": 4 * 2.0 ** -11, "bf16": 4 * 2.0 ** -8}[form]
        if case == "window_fallback":
            # a few pairs per bin: the per-element rounding bound of the form (operand
            # rounding plus FP32 accumulation over K = 3 T0 terms and the tile's bin sums)
            per = {"split_bf16": 3 * 2.0 ** -16, "tf32": 2 * 2.0 ** -11}[form]
            bound = per + (3 * T0 + 256) * 2.0 ** -24
            assert oracle.rounding_ratio(C0[:, :nb], ref).max() <= bound
        else:
            assert oracle.bin_error(C0[:, :nb], ref).max() <= tol
        if q is not None:
            assert oracle.phase_error(S0[..., 0], ref, "cos").max() <= tol
            if sine:
                assert oracle.phase_error(S0[..., 1], ref, "sin").max() <= tol


def test_batched_order_invariant(asd):
    """Three problems in one batched launch, submitted in two orders: each problem's
    sums are bit for bit the same (the work list and the schedule differ)."""
    lats = [synth.hypercubic(L, d, True) for L, d in ((40, 2), (11, 3), (23, 2))]
    T0, n_t = 20, 5
    trs = [synth.traj_precess(l.n_sites, T0 + n_t, seed=50 + k) for k, l in enumerate(lats)]

    def once(order):
        plans, ds, Cs = [], [], []
        for k in order:
            lat = lats[k]
            w = 1.0 if lat.coords[:, 2].max() == 0 else 0.5
            nb = 12
            plans.append(asd.CorrPlan.for_lattice(lat, T0 + n_t, T0, n_t, w, nb,
                                                  precision="split_bf16", tile_n=256,
                                                  deterministic=True))
            ds.append(torch.from_numpy(np.ascontiguousarray(trs[k])).cuda())
            Cs.append(torch.zeros((n_t, nb), dtype=torch.float64, device="cuda"))
        asd.pair_corr_batched(plans, ds, Cs)
        assert asd.sync_status() == 0
        for p in plans:
            p.close()
        return {k: C.cpu().numpy() for k, C in zip(order, Cs)}

    a, b = once([0, 1, 2]), once([2, 0, 1])
    for k in range(3):
        assert bits_equal(a[k], b[k]), f"problem {k} differs with the batch order"
        lat = lats[k]
        w = 1.0 if lat.coords[:, 2].max() == 0 else 0.5
        ref = oracle.pair_corr(trs[k], T0, list(range(n_t)), oracle.Geometry.of_lattice(lat),
                               w, 12)
        assert oracle.bin_error(a[k], ref).max() <= 1e-5


def test_rejects_mixed_batch(asd):
    lat = synth.hypercubic(10, 2, True)
    p1 = asd.CorrPlan.for_lattice(lat, 12, 8, 3, 1.0, 5, tile_n=256, deterministic=True)
    p2 = asd.CorrPlan.for_lattice(lat, 12, 8, 3, 1.0, 5, tile_n=256)
    tr = torch.from_numpy(synth.traj_iid(lat.n_sites, 12, seed=1)).cuda()
    C = [torch.zeros((3, 5), dtype=torch.float64, device="cuda") for _ in range(2)]
    with pytest.raises(asd.AsdError):
        asd.pair_corr_batched([p1, p2], [tr, tr], C)
    p1.close()
    p2.close()
