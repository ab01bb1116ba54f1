"""Failure detection without a GPU fault: a bounded wait that nothing satisfies gives up,
the host reads ASD_ETIMEOUT from the device error word, and the same context then runs
the hot path correctly."""
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


def test_bounded_wait_times_out_and_context_survives(asd):
    assert asd.sync_status() == asd.ASD_OK
    asd.selftest_timeout(20_000_000)                 # 20 ms
    assert asd.sync_status() == asd.ASD_ETIMEOUT
    assert asd.sync_status() == asd.ASD_OK           # reported once, then cleared
    with pytest.raises(asd.AsdError):
        asd.selftest_timeout(0)                      # limit out of range, nothing launched

    lat = synth.hypercubic(6, 3, True)
    tr = synth.traj_precess(lat.n_sites, 20, seed=4)
    plan = asd.CorrPlan.for_lattice(lat, 20, 12, 4, 0.5, 12, precision="split_bf16")
    C = torch.zeros((4, 12), dtype=torch.float64, device="cuda")
    plan.run(torch.from_numpy(np.ascontiguousarray(tr[:, None])).cuda(), C)
    assert asd.sync_status() == asd.ASD_OK
    ref = oracle.pair_corr(tr, 12, list(range(4)), oracle.Geometry.of_lattice(lat), 0.5, 12)
    assert oracle.bin_error(C.cpu().numpy(), ref).max() <= 1e-5
    plan.close()
