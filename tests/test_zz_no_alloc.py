"""asd_ll_integrate_noalloc: the LL integrator for callers that cannot allocate device
memory (a global-mode stream capture on another thread, a process whose device memory
belongs to its own pool, a loop that cannot take cudaMalloc's implicit synchronisation).
Its work buffers live in a fixed device array reserved with the library.

It must reproduce asd_ll_integrate (same kernels, same arithmetic, so within the
tolerance of the LL parity test: here it is bit-identical) on two calls in a row --
the second call reuses the array the first one left behind -- and refuse requests
larger than its fixed area.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2308_07487_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asd():
    from paper_2308_07487_gb300 import asd as m
    return m


def _run(asd, fn, sysm, s0, F, stride):
    S, N = s0.shape[0], s0.shape[1]
    traj = torch.full((N, S, F, 3), float("nan"), dtype=torch.float32, device="cuda")
    out = torch.full_like(s0, float("nan"))
    rc = fn(ctypes.byref(sysm.c), S, s0.data_ptr(), 0.01, F, stride, traj.data_ptr(),
            out.data_ptr(), None)
    assert rc == 0, asd.strerror(rc)
    assert asd.sync_status() == 0
    return traj.cpu().numpy(), out.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(asd):
    lat = synth.hypercubic(12, 3, True, J=-1.0, Hz=0.5)
    sysm = asd.System(lat)
    S, F, stride = 3, 25, 2
    for call, seed in enumerate((41, 42)):
        s0 = torch.from_numpy(synth.random_unit(S * lat.n_sites, seed)
                              .reshape(S, lat.n_sites, 3)).cuda()
        ref_tr, ref_out = _run(asd, asd.lib.asd_ll_integrate, sysm, s0, F, stride)
        got_tr, got_out = _run(asd, asd.lib.asd_ll_integrate_noalloc, sysm, s0, F, stride)
        assert np.isfinite(got_tr).all() and np.isfinite(got_out).all()
        assert np.abs(got_tr - ref_tr).max() <= 2e-5, f"call {call}"
        assert np.abs(got_out - ref_out).max() <= 2e-5, f"call {call}"


def test_noalloc_refuses_requests_beyond_its_fixed_area(asd):
    lat = synth.hypercubic(64, 3, True)          # 262144 sites
    sysm = asd.System(lat)
    s0 = torch.zeros((2, lat.n_sites, 3), dtype=torch.float32, device="cuda")
    traj = torch.zeros((lat.n_sites, 2, 2, 3), dtype=torch.float32, device="cuda")
    rc = asd.lib.asd_ll_integrate_noalloc(ctypes.byref(sysm.c), 2, s0.data_ptr(), 0.01, 2, 1,
                                          traj.data_ptr(), None, None)
    assert rc == asd.ASD_EINVAL
    assert "262144" in asd.strerror(rc)
