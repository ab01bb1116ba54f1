"""CTA pairs (asd_corr_desc.cta_pair, tcgen05 cta_group::2): 256-row tiles over two SMs,
each CTA loading its 128 A rows and half of the B columns.  Parity against the FP64 oracle
for the lattice table path, the position path with bins and phase weights (both parts, K
chunks, rows from mid-tile), the BF16 and TF32 forms; the deterministic mode gives the
same sums as one CTA per tile (each CTA's half of a pair tile is a one-CTA tile); plans
that cannot use pairs are refused.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"split_bf16": 1e-5, "tf32": 4 * 2.0 ** -11, "bf16": 4 * 2.0 ** -8}


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def run(asd, lat, tr, T0, n_t, w, nb, form, q=None, sine=False, rows=None, **kn):
    F = tr.shape[-2]
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision=form, q=q,
                                    phase_sine=sine, **kn)
    d = torch.from_numpy(np.ascontiguousarray(tr)).cuda()
    C = torch.zeros((n_t, max(nb, 1)), dtype=torch.float64, device="cuda")
    nq = 0 if q is None else len(q)
    Sq = torch.zeros((n_t, max(nq, 1), 1 + int(sine)), dtype=torch.float64, device="cuda")
    plan.run(d, C if nb else None, Sq if nq else None, rows=rows)
    assert asd.sync_status() == 0
    plan.close()
    return C.cpu().numpy()[:, :nb], Sq.cpu().numpy()


@pytest.mark.parametrize("form", ["split_bf16", "bf16", "tf32"])
def test_lattice_pairs(asd, form):
    """Periodic 3D lattice (N = 4913 > 4096: 256-wide tiles), rows from mid-tile (a
    ragged last pair tile whose second CTA has no rows left)."""
    lat = synth.hypercubic(17, 3, True)
    T0, n_t, w, nb = 40, 5, 0.5, 30
    tr = synth.traj_precess(lat.n_sites, T0 + n_t, seed=71)
    rows = (70, 4700)
    C, _ = run(asd, lat, tr, T0, n_t, w, nb, form, rows=rows, cta_pair=True)
    ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb,
                           rows=rows)
    assert oracle.bin_error(C, ref).max() <= TOL[form]


@pytest.mark.parametrize("form", ["split_bf16", "bf16"])
def test_glass_pairs_bins_and_phase(asd, form):
    """Jittered +-J glass (FP32 positions), 8 epilogue warps, 192-wide tiles, bins and 13
    q-vectors with the sine part, two K chunks, rows from mid-tile."""
    lat = synth.hypercubic(20, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 4),
                           jitter=0.1)
    q = synth.q_vectors_glass()[::5]
    T0, n_t, w, nb = 64, 4, 0.5, 60
    tr = synth.traj_precess(lat.n_sites, T0 + n_t, seed=72)
    rows = (300, 5100)
    C, S = run(asd, lat, tr, T0, n_t, w, nb, form, q=q, sine=True, rows=rows, cta_pair=True,
               k_chunks=2)
    ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb,
                           q=q, rows=rows)
    assert oracle.bin_error(C, ref).max() <= TOL[form]
    assert oracle.phase_error(S[..., 0], ref, "cos").max() <= TOL[form]
    assert oracle.phase_error(S[..., 1], ref, "sin").max() <= TOL[form]


def test_pairs_match_single_cta_in_deterministic_mode(asd):
    """Each CTA of a pair bins the same 128 x BN tile a single CTA would: with fixed-point
    sums the two layouts agree to the last unit of the fixed-point scale."""
    lat = synth.hypercubic(18, 3, True)
    T0, n_t, w, nb = 30, 4, 0.5, 25
    tr = synth.traj_precess(lat.n_sites, T0 + n_t, seed=73)
    a, _ = run(asd, lat, tr, T0, n_t, w, nb, "split_bf16", deterministic=True, tile_n=256)
    b, _ = run(asd, lat, tr, T0, n_t, w, nb, "split_bf16", deterministic=True, tile_n=256,
               cta_pair=True)
    ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb)
    m = ref["M_abs"] > 0
    assert (np.abs(a - b)[m] / ref["M_abs"][m]).max() <= 1e-12
    assert oracle.bin_error(b, ref).max() <= 1e-5


def test_pair_refusals(asd):
    lat = synth.hypercubic(12, 2, True)
    with pytest.raises(asd.AsdError):
        asd.CorrPlan.for_lattice(lat, 12, 8, 3, 1.0, 5, precision="fp32", cta_pair=True)
    with pytest.raises(asd.AsdError):
        asd.CorrPlan.for_lattice(lat, 12, 8, 3, 1.0, 5, tile_n=128, cta_pair=True)
    p = asd.CorrPlan.for_lattice(lat, 12, 8, 3, 1.0, 5, tile_n=256, cta_pair=True)
    tr = torch.from_numpy(synth.traj_iid(lat.n_sites, 12, seed=1)).cuda()
    C = torch.zeros((3, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(asd.AsdError):
        asd.pair_corr_batched([p], [tr], [C])
    p.close()
