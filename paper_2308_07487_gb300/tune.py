"""Autotuner of the tensor-core pair-correlation launch.

The launch knobs of a plan -- tile width (`tile_n`), epilogue warps (`epi_warps`), raster
group height (`raster_m`), pipeline stages (`stages`) and CTA pairs (`cta_pair`, single
problems only) -- change speed, and results only through the rounding order of the FP32
per-tile bin sums and of the FP64 accumulation.
(`k_chunks` also changes the tensor core's accumulation error, so it stays at the plan's
accuracy-driven default and is not tuned.)
The tuner times each valid candidate on a sample of the workload (a few displacements)
with CUDA events and keeps the fastest; results are cached in memory and, when a path is
given, in a JSON file keyed by the problem's shape, so later runs skip the timing.

For a batch, every problem of one launch shares the tile width and warp count, so the
batch is tuned as a whole (on plans built with the sample's displacement count).
"""
from __future__ import annotations

import itertools
import json
import os

DEFAULT_SPACE = {
    "tile_n": [128, 192, 256],
    "epi_warps": [4, 8],
    "raster_m": [8, 16, 32, 64],
    "stages": [0, 3],
    "cta_pair": [False, True],
}


def candidates(space=None, n_q=0, N=None, batch=False):
    """Valid combinations of the knobs (the plan's instantiated kernels): 128-wide tiles
    run with 4 epilogue warps; with phase weights (n_q > 0) the phase product takes 128
    TMEM columns beside the two accumulators, so tiles are at most 192 wide; tiles wider
    than the problem are skipped; CTA pairs need 192- or 256-wide tiles and a single
    problem (not a batch)."""
    sp = dict(DEFAULT_SPACE if space is None else space)
    out = []
    keys = sorted(sp)
    for vals in itertools.product(*(sp[k] for k in keys)):
        c = dict(zip(keys, vals))
        tn, ew = c.get("tile_n", 0), c.get("epi_warps", 4)
        if tn == 128 and ew != 4:
            continue
        if n_q > 0 and tn == 256:
            continue
        if N is not None and tn and tn > 128 and N <= 128:
            continue
        if c.get("cta_pair") and (batch or tn == 128):
            continue
        out.append(c)
    return out


def problem_key(kind, precision, shapes):
    """Cache key: the form and the shapes that decide the best launch."""
    return f"{kind}|{precision}|" + ";".join(
        "N{N},S{S},K{K},nb{nb},nq{nq},g{g}".format(**s) for s in shapes)


def shape_of(lat, T0, S, n_bins, n_q):
    jittered = not (lat.pos == lat.coords).all()
    return {"N": int(lat.n_sites), "S": int(S), "K": int(3 * T0), "nb": int(n_bins),
            "nq": int(n_q), "g": "pos" if jittered else ("per" if lat.periodic else "open")}


class Tuner:
    """Timing-based selection with a cache.  `timer(fn)` returns seconds per call of fn
    (the default times CUDA work with events after one untimed call)."""

    def __init__(self, path=None, timer=None, reps=2):
        self.path = path
        self.reps = reps
        self.timer = timer or self._cuda_timer
        self.cache = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    def _cuda_timer(self, fn):
        import torch
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(self.reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / self.reps

    def _save(self):
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def select(self, key, cands, run):
        """Best of `cands` by `run(cand) -> seconds` (cached under `key`)."""
        if key in self.cache:
            return dict(self.cache[key]["best"])
        timings = []
        for c in cands:
            try:
                t = run(c)
            except Exception:          # a combination the plan rejects (e.g. no fit)
                continue
            timings.append((t, c))
        if not timings:
            raise RuntimeError("autotune: no candidate ran")
        t, best = min(timings, key=lambda x: x[0])
        self.cache[key] = {"best": best, "seconds": t,
                           "tried": [{"cand": c, "seconds": s} for s, c in timings]}
        self._save()
        return dict(best)

    # -- single problem -------------------------------------------------------------
    def tune_plan(self, asd, lat, F, T0, w, n_bins, traj, precision="split_bf16", S=1, q=None,
                  n_t_sample=4, space=None, center=False):
        """Best knobs for asd.CorrPlan.for_lattice(...) on this problem, timed on the
        contraction of `n_t_sample` displacements of the prepared trajectory."""
        n_q = 0 if q is None else len(q)
        key = problem_key("plan", precision, [shape_of(lat, T0, S, n_bins, n_q)])

        def run(c):
            import torch
            plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t_sample, w, n_bins,
                                            precision=precision, S=S, q=q, center=center, **c)
            try:
                C = torch.zeros((n_t_sample, max(n_bins, 1)), dtype=torch.float64,
                                device="cuda") if n_bins else None
                Sq = torch.zeros((n_t_sample, n_q), dtype=torch.float64,
                                 device="cuda") if n_q else None
                plan.prepare(traj)
                return self.timer(lambda: plan.contract(C, Sq))
            finally:
                plan.close()
        return self.select(key, candidates(space, n_q, lat.n_sites), run)

    # -- batch ----------------------------------------------------------------------
    def tune_batch(self, asd, problems, F, T0, trajs, precision="split_bf16", n_t_sample=4,
                   space=None):
        """Best shared knobs for one batched launch over `problems` = [(lat, w, n_bins)]."""
        shapes = [shape_of(lat, T0, 1, nb, 0) for lat, w, nb in problems]
        key = problem_key("batch", precision, shapes)

        def run(c):
            import torch
            plans = [asd.CorrPlan.for_lattice(lat, F, T0, n_t_sample, w, nb,
                                              precision=precision, **c)
                     for lat, w, nb in problems]
            try:
                Cs = [torch.zeros((n_t_sample, nb), dtype=torch.float64, device="cuda")
                      for _, _, nb in problems]
                return self.timer(lambda: asd.pair_corr_batched(plans, trajs, Cs))
            finally:
                for p in plans:
                    p.close()
        return self.select(key, candidates(space, 0, min(l.n_sites for l, _, _ in problems),
                                           batch=True), run)
