"""asd_pair_corr_normalize (Eq. 3's 1/N and the average of Eq. 4) against oracle.normalize:
C(b,t) = C_sum / (S T0 n_b) with 0 in empty bins, S(q,t) = Sq_sum / (N S T0) for the
cosine and the sine part, element by element at 1e-12 relative, on the library's own
sums; then the normalised result of the whole path against the normalised oracle."""
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


@pytest.fixture(scope="module")
def case(asd):
    """7^3 periodic lattice (w = 0.5: no lattice distance in [0.5, 1), so bin 1 is
    empty), S = 2 samples, 9 displacements, 13 q with cosine and sine parts."""
    lat = synth.hypercubic(7, 3, True)
    tr = synth.traj_precess(lat.n_sites, 30, seed=31, S=2)
    q = synth.q_vectors_glass()[::5]
    T0, n_t, w, nb = 18, 9, 0.5, 11
    plan = asd.CorrPlan.for_lattice(lat, 30, T0, n_t, w, nb, precision="split_bf16", S=2,
                                    q=q, phase_sine=True)
    C = torch.zeros((n_t, nb), dtype=torch.float64, device="cuda")
    Sq = torch.zeros((n_t, len(q), 2), dtype=torch.float64, device="cuda")
    plan.run(torch.from_numpy(np.ascontiguousarray(tr)).cuda(), C, Sq)
    assert asd.sync_status() == 0
    ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb,
                           q=q)
    yield dict(plan=plan, C_sum=C, Sq_sum=Sq, ref=ref, lat=lat)
    plan.close()


def _oracle_norm(C_sum, Sq_part, ref):
    """oracle.normalize applied to given sums (the library's), with the oracle's counts."""
    res = dict(ref)
    res["C_sum"], res["Sq_sum"] = C_sum, Sq_part
    return oracle.normalize(res)


def test_normalize_matches_oracle_normalize(asd, case):
    plan, C_sum, Sq_sum, ref = case["plan"], case["C_sum"], case["Sq_sum"], case["ref"]
    counts = plan.counts()
    np.testing.assert_array_equal(counts, ref["counts"])
    assert (counts == 0).any() and (counts > 0).any()     # empty bins are exercised
    C = torch.full_like(C_sum, np.nan)
    Sq = torch.full_like(Sq_sum, np.nan)
    plan.normalize(C_sum, Sq_sum, C, Sq)
    assert asd.sync_status() == 0
    cs, sq = C_sum.cpu().numpy(), Sq_sum.cpu().numpy()
    for part in (0, 1):
        Cr, Sr = _oracle_norm(cs, sq[..., part], ref)
        np.testing.assert_allclose(Sq.cpu().numpy()[..., part], Sr, rtol=1e-12, atol=0)
    np.testing.assert_allclose(C.cpu().numpy(), Cr, rtol=1e-12, atol=0)
    assert not C.cpu().numpy()[:, counts == 0].any()      # 0, not NaN, in empty bins


def test_normalize_in_place_and_one_output(asd, case):
    """C may alias C_sum and Sq may alias Sq_sum; either pair may be NULL."""
    plan, ref = case["plan"], case["ref"]
    C = case["C_sum"].clone()
    Sq = case["Sq_sum"].clone()
    expect_c = torch.empty_like(C)
    expect_q = torch.empty_like(Sq)
    plan.normalize(C, Sq, expect_c, expect_q)
    plan.normalize(C, Sq, C, Sq)                       # in place
    assert asd.sync_status() == 0
    assert torch.equal(C, expect_c) and torch.equal(Sq, expect_q)
    only_c = torch.empty_like(C)
    plan.normalize(case["C_sum"], None, only_c, None)
    only_q = torch.empty_like(Sq)
    plan.normalize(None, case["Sq_sum"], None, only_q)
    assert asd.sync_status() == 0
    assert torch.equal(only_c, expect_c) and torch.equal(only_q, expect_q)
    with pytest.raises(asd.AsdError):
        plan.normalize(case["C_sum"], None, None, None)   # a sum without its output


def test_normalized_path_matches_normalized_oracle(asd, case):
    """C(b,t) and S(q,t) of the whole path (split-BF16 sums, then the library's
    normalisation) against oracle.normalize of the oracle's sums: |dC| <= 1e-5 M_abs /
    (S T0 n_b) per bin, |dS| <= 1e-5 Sq_abs / (N S T0) per (t, q)."""
    plan, ref = case["plan"], case["ref"]
    C = torch.empty_like(case["C_sum"])
    Sq = torch.empty_like(case["Sq_sum"])
    plan.normalize(case["C_sum"], case["Sq_sum"], C, Sq)
    assert asd.sync_status() == 0
    Cr, Sr = oracle.normalize(ref)
    n = ref["counts"].astype(np.float64)
    S, T0, N = ref["S"], ref["T0"], ref["N"]
    occ = n > 0
    dC = np.abs(C.cpu().numpy() - Cr)[:, occ]
    assert (dC <= 1e-5 * ref["M_abs"][:, occ] / (S * T0 * n[occ]) + 1e-300).all()
    dS = np.abs(Sq.cpu().numpy()[..., 0] - Sr)
    assert (dS <= 1e-5 * ref["Sq_abs"] / (N * S * T0) + 1e-300).all()
    # C(0, 0) = 1 for unit spins: bin 0 holds the self pairs only on a lattice
    assert abs(C.cpu().numpy()[0, 0] - 1.0) <= 1e-5
