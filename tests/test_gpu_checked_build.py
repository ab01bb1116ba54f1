"""The index-checked build (ASD_CHECK_BOUNDS=1, libasd_checked.so): it stands in for a
memory checker.  In a child process that loads it (ASD_CHECKED=1), every kernel path of
the contraction runs on small cases -- lattice table and threshold paths, the branch-free
position path, the private window with fallback bins, the tensor-core phase product with
its sine part, K-chunks, the FP32 form, CTA pairs, tiles binned through two windows, a
batched launch -- with no index check failing (asd_sync_status == ASD_OK) and results at the parity bar of the oracle; the self-test
makes one check fail on purpose (no memory is touched) and must read back ASD_EBOUNDS.
In the normal build the self-test is refused.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, numpy as np, torch
import oracle
from paper_2308_07487_gb300 import asd, synth
assert asd.build_flags() & asd.ASD_BUILD_CHECK_BOUNDS
out = {}
asd.selftest_bounds()
out["selftest"] = asd.sync_status()
out["after_selftest"] = asd.sync_status()

def case(name, lat, T0, n_t, w, nb, form, q=None, sine=False, rows=None, **kn):
    F = T0 + n_t + 1
    tr = synth.traj_precess(lat.n_sites, F, seed=61)
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision=form, q=q,
                                    phase_sine=sine, **kn)
    d = torch.from_numpy(np.ascontiguousarray(tr)).cuda()
    C = torch.zeros((n_t, max(nb, 1)), dtype=torch.float64, device="cuda")
    nq = 0 if q is None else len(q)
    Sq = torch.zeros((n_t, max(nq, 1), 1 + int(sine)), dtype=torch.float64, device="cuda")
    plan.run(d, C if nb else None, Sq if nq else None, rows=rows)
    st = asd.sync_status()
    plan.close()
    ref = oracle.pair_corr(tr, T0, list(range(n_t)), oracle.Geometry.of_lattice(lat), w, nb,
                           q=q, rows=rows)
    c = C.cpu().numpy()[:, :nb]
    r = {"status": st}
    if nb:
        r["bin"] = float(oracle.bin_error(c, ref).max())
        r["round"] = float(oracle.rounding_ratio(c, ref).max())
    if nq:
        r["phase"] = float(oracle.phase_error(Sq.cpu().numpy()[..., 0], ref, "cos").max())
        if sine:
            r["phase_sin"] = float(oracle.phase_error(Sq.cpu().numpy()[..., 1], ref, "sin").max())
    out[name] = r

glass = synth.hypercubic(12, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 4), jitter=0.1)
case("lattice_lut", synth.hypercubic(13, 3, True), 20, 4, 0.5, 19, "split_bf16")
case("lattice_thr_rows", synth.hypercubic(100, 2, False), 16, 4, 1.0, 57, "split_bf16",
     rows=(50, 900))
case("lattice_window", synth.hypercubic(9, 3, True), 16, 3, 0.0125, 640, "split_bf16")
case("lattice_bf16_256", synth.hypercubic(11, 3, True), 16, 3, 0.5, 17, "bf16", tile_n=256)
case("positions_phase", glass, 48, 4, 0.5, 36, "split_bf16", q=synth.q_vectors_glass()[::6],
     sine=True, rows=(21, 900), k_chunks=2)
case("positions_ew8", glass, 48, 3, 0.5, 36, "tf32", tile_n=192, epi_warps=8)
case("window_fallback", synth.hypercubic(8, 3, False, jitter=0.1, seed=4, block=(4, 4, 2)),
     12, 3, 0.01, 1500, "split_bf16")
case("fp32_phase", glass, 32, 3, 0.5, 36, "fp32", q=synth.q_vectors_glass()[::9], sine=True)
case("deterministic", glass, 32, 3, 0.5, 36, "split_bf16", q=synth.q_vectors_glass()[::9],
     deterministic=True)
case("pair_phase", glass, 32, 3, 0.5, 36, "split_bf16", q=synth.q_vectors_glass()[::9],
     rows=(40, 1700), cta_pair=True)
case("pair_lattice", synth.hypercubic(17, 3, True), 20, 3, 0.5, 30, "split_bf16", cta_pair=True)
glass32 = synth.hypercubic(32, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 8), jitter=0.1)
case("positions_two_windows", glass32, 32, 2, 0.5, 256, "split_bf16",
     q=synth.q_vectors_glass()[::8], rows=(0, 256))
lats = [synth.hypercubic(L, 2, True) for L in (30, 17)]
plans = [asd.CorrPlan.for_lattice(l, 14, 12, 3, 1.0, 10, tile_n=256) for l in lats]
trs = [torch.from_numpy(synth.traj_precess(l.n_sites, 14, seed=3)).cuda()
       for l in lats]
Cs = [torch.zeros((3, 10), dtype=torch.float64, device="cuda") for _ in lats]
asd.pair_corr_batched(plans, trs, Cs)
out["batched"] = {"status": asd.sync_status()}
for p in plans:
    p.close()
print("RESULT " + json.dumps(out))
'''


def test_checked_build_paths():
    sys.path.insert(0, ROOT)
    from paper_2308_07487_gb300 import build
    build.build(check_bounds=True)
    env = dict(os.environ, ASD_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    from paper_2308_07487_gb300 import asd
    assert out.pop("selftest") == asd.ASD_EBOUNDS
    assert out.pop("after_selftest") == asd.ASD_OK  # the word was cleared
    tol = {"bf16": 4 * 2.0 ** -8, "tf32": 4 * 2.0 ** -11}
    for name, res in out.items():
        assert res["status"] == asd.ASD_OK, (name, res)
        t = tol["bf16"] if "bf16_" in name else tol["tf32"] if "ew8" in name else 1e-5
        if name in ("window_fallback", "lattice_window"):
            assert res["round"] <= 3 * 2.0 ** -16 + 300 * 2.0 ** -24, (name, res)
        elif "bin" in res:
            assert res["bin"] <= t, (name, res)
        for k in ("phase", "phase_sin"):
            if k in res:
                assert res[k] <= t, (name, res)


def test_normal_build_refuses_bounds_selftest():
    from paper_2308_07487_gb300 import asd
    if asd.build_flags() & asd.ASD_BUILD_CHECK_BOUNDS:
        pytest.skip("this process loaded the checked build")
    with pytest.raises(asd.AsdError) as e:
        asd.selftest_bounds()
    assert e.value.status == asd.ASD_EUNSUPPORTED
