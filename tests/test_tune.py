"""Host logic of the launch autotuner (no GPU): candidate filtering, cache keys, selection
and the JSON cache round trip, with a fake timer."""
import json

from paper_2308_07487_gb300 import synth, tune


def test_candidates_respect_the_instantiated_kernels():
    cs = tune.candidates()
    assert cs and all(not (c["tile_n"] == 128 and c["epi_warps"] != 4) for c in cs)
    # with phase weights the phase product needs 128 TMEM columns: tiles of at most 192
    # columns (either warp count at 192)
    cq = tune.candidates(n_q=8)
    assert cq and {c["tile_n"] for c in cq} == {128, 192}
    assert {c["epi_warps"] for c in cq if c["tile_n"] == 192} == {4, 8}
    assert all(c["tile_n"] == 128 for c in tune.candidates(N=100))
    # CTA pairs: 192- or 256-wide tiles, never for a batch
    assert any(c.get("cta_pair") for c in cs)
    assert all(c["tile_n"] != 128 for c in cs if c.get("cta_pair"))
    assert not any(c.get("cta_pair") for c in tune.candidates(batch=True))
    # every combination appears once
    assert len({json.dumps(c, sort_keys=True) for c in cs}) == len(cs)


def test_problem_key_distinguishes_shapes():
    a = synth.hypercubic(6, 3, True)
    b = synth.hypercubic(6, 3, False)
    ka = tune.problem_key("plan", "split_bf16", [tune.shape_of(a, 16, 1, 9, 0)])
    kb = tune.problem_key("plan", "split_bf16", [tune.shape_of(b, 16, 1, 9, 0)])
    kc = tune.problem_key("plan", "bf16", [tune.shape_of(a, 16, 1, 9, 0)])
    assert len({ka, kb, kc}) == 3
    assert ka == tune.problem_key("plan", "split_bf16", [tune.shape_of(a, 16, 1, 9, 0)])


def test_select_picks_fastest_skips_rejected_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    t = tune.Tuner(path=path, timer=lambda fn: fn())
    cands = [{"tile_n": 128}, {"tile_n": 256}, {"tile_n": 512}]
    calls = []

    def run(c):
        calls.append(c["tile_n"])
        if c["tile_n"] == 512:
            raise RuntimeError("rejected by the plan")
        return {128: 2.0, 256: 1.0}[c["tile_n"]]

    assert t.select("k", cands, run) == {"tile_n": 256}
    assert calls == [128, 256, 512]
    # cached: no new timing, also from a fresh tuner reading the file
    assert t.select("k", cands, run) == {"tile_n": 256}
    t2 = tune.Tuner(path=path, timer=lambda fn: fn())
    assert t2.select("k", cands, lambda c: 1 / 0) == {"tile_n": 256}
    assert len(calls) == 3
    rec = json.load(open(path))["k"]
    assert rec["seconds"] == 1.0 and len(rec["tried"]) == 2
