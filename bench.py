#!/usr/bin/env python3
"""Benchmark of the fused pair-correlation hot path on GB300.

Default workload (the precision-sweep configuration): 64^3 = 262144 spins at simple-cubic
positions with Gaussian jitter sigma = 0.1, open boundaries, +-J couplings (p = 0.5),
thermalised at T = 1.0 J (Metropolis, adaptive cone); LL RK4 with dt = 0.01 and F = 640
frames; C(r,t) over T0 = 512 origins in 256 distance bins of width 0.5 plus S(q,t) for 64
q-vectors (cos(q.r_ij) weights), 128 displacements.  Contraction per displacement:
N x N x 3*T0 (K = 1536), about 2.1e14 flops.

One step = the hot path on one batch: the LL trajectory from the resident thermalised
spins (asd_ll_integrate), operand preparation, the fused contraction with the binning and
phase epilogues over one block of displacements (asd_pair_corr_contract_range; the step
index picks the block, so consecutive steps walk through all 128 displacements), and
normalisation (asd_pair_corr_normalize).  Every displacement costs the same, so a step
is a fixed amount of work: n_t_per_step * 2 N^2 K flops.
Metric: algorithmic contraction TFLOP/s = n_t_per_step * 2 N^2 (3 T0) / step time.

--workload cubic40 runs the 40^3 periodic lattice (N = 64000, K = 3000, 200
displacements, 70 bins, all displacements per step); ensemble and learned print their
own lines.  --impl reference runs the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused pair-corr TFLOP/s & % tensor peak, split-BF16 vs FP32 at ≤1e-5 rel err"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="split_bf16", choices=["split_bf16", "bf16", "tf32", "fp32"])
    ap.add_argument("--small", action="store_true", help="tiny workload (smoke)")
    ap.add_argument("--medium", action="store_true", help="profiling workload (ncu)")
    ap.add_argument("--no-extras", action="store_true", help="skip form sweep, CPU baseline, e2e")
    ap.add_argument("--ncu", action="store_true", help="one step, nothing else (for ncu)")
    ap.add_argument("--mlp-depth", type=int, default=2, choices=[2, 3],
                    help="learned workload: hidden layers of the proposal network")
    ap.add_argument("--cta-pair", action="store_true",
                    help="CTA pairs (cta_group::2) for the timed contraction (tensor forms)")
    ap.add_argument("--nt-per-step", type=int, default=0,
                    help="displacements per step (0: the workload's default)")
    ap.add_argument("--workload", default="glass64",
                    choices=["glass64", "cubic40", "ensemble", "learned", "kernels"],
                    help="glass64: the headline line; cubic40 its own line; the others "
                         "print their own lines (kernels: one small launch of every other "
                         "kernel, for per-kernel profiles)")
    return ap.parse_args()


def workload(name, small=False, medium=False):
    """Sizes of one bench workload.  nt_step = displacements per step."""
    from paper_2308_07487_gb300 import synth
    if name == "glass64":
        if medium:
            # profiling case of the same kernel shapes (K, bins, q): 32^3 glass, 2 displacements
            lat = synth.hypercubic(32, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 8),
                                   jitter=0.1)
            return dict(name="glass32_open_N32768", lat=lat, F=640, T0=512, n_t=2, w=0.5,
                        n_bins=256, q=synth.q_vectors_glass(), T=1.0, sweeps=50, dt=0.01,
                        nt_step=2)
        if small:
            lat = synth.hypercubic(16, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 8),
                                   jitter=0.1)
            return dict(name="glass16_open_N4096", lat=lat, F=160, T0=128, n_t=32, w=0.5,
                        n_bins=256, q=synth.q_vectors_glass(), T=1.0, sweeps=50, dt=0.01,
                        nt_step=8)
        cfg = synth.cfg_glass64()
        return dict(name=cfg.name, lat=cfg.lattice, F=cfg.F, T0=cfg.T0, n_t=cfg.n_t, w=cfg.w,
                    n_bins=cfg.n_bins, q=cfg.q, T=cfg.T, sweeps=200, dt=0.01, nt_step=8)
    if medium:
        # profiling case: same K and bin width as the throughput workload, 26^3 sites,
        # 4 displacements (operands ~2 GB: larger than L2, small enough for ncu replay)
        lat = synth.hypercubic(26, 3, True, J=1.0, seed=23082)
        return dict(name="sc26_periodic_N17576", lat=lat, F=1003, T0=1000, n_t=4, w=0.5,
                    n_bins=46, q=None, T=1.2, sweeps=200, dt=0.01, nt_step=4)
    if small:
        lat = synth.hypercubic(16, 3, True, J=1.0, seed=23082)
        return dict(name="sc16_periodic_N4096", lat=lat, F=160, T0=128, n_t=32, w=0.5, n_bins=28,
                    q=None, T=1.2, sweeps=200, dt=0.01, nt_step=32)
    cfg = synth.cfg_cubic40()
    return dict(name=cfg.name, lat=cfg.lattice, F=cfg.F, T0=cfg.T0, n_t=cfg.n_t, w=cfg.w,
                n_bins=cfg.n_bins, q=None, T=cfg.T, sweeps=2000, dt=0.01, nt_step=cfg.n_t)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 7:
                self.samples.append(p)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x):
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# -------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample of the same workload
# -------------------------------------------------------------------------------------
def oracle_rows(threads):
    """Rows of an oracle sample: the oracle runs its OpenMP loop over rows, so four rows
    per thread (at least 64) keep every thread busy."""
    return max(64, 4 * threads)


def oracle_sample(W, tr_np, rows, t_list):
    """The FP64 oracle on rows [rows) x all columns at the displacements t_list, with
    the workload's bins and q-vectors; flops counted like the GPU's (2 N_rows N K per
    displacement)."""
    import oracle
    geo = oracle.Geometry.of_lattice(W["lat"])
    t0 = time.perf_counter()
    res = oracle.pair_corr(tr_np, W["T0"], t_list, geo, W["w"], W["n_bins"], q=W["q"],
                           rows=rows)
    dt = time.perf_counter() - t0
    N = W["lat"].n_sites
    flops = 2.0 * (rows[1] - rows[0]) * N * len(t_list) * 3 * W["T0"]
    return res, dt, flops


def run_reference(args, W, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2308_07487_gb300 import synth
    if ws > 1:
        # the other ranks do no work: rank 0 takes every CPU of the process, as at one GPU
        # (the launcher pins each rank to one OpenMP thread)
        oracle.set_threads(len(os.sched_getaffinity(0)))
    N = W["lat"].n_sites
    tr = synth.traj_precess(N, W["F"], seed=23082)
    threads = oracle.threads()
    rows = (0, min(N, oracle_rows(threads)))
    t_list = [0, W["n_t"] - 1]
    oracle_sample(W, tr, (0, 1), [0])  # warm the OpenMP pool
    times, flops = [], 0.0
    for _ in range(args.warmup):
        oracle_sample(W, tr, rows, t_list)
    for _ in range(args.steps):
        _, dt, flops = oracle_sample(W, tr, rows, t_list)
        times.append(dt)
    t = max(times)
    v = flops / t / 1e12
    cores = min(threads, rows[1] - rows[0])
    sample = (f"rows {rows[0]}..{rows[1]} x all {N} columns x t in {t_list} (K = {3 * W['T0']}, "
              f"{W['n_bins']} bins, {0 if W['q'] is None else len(W['q'])} q)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": W["name"], "sample": sample},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def measured_extra_peaks():
    """TF32 tensor and FP32 (FFMA) GEMM rates of this GPU through cuBLAS (torch.matmul,
    8192^3, best of 5 after a warm-up): the denominators of the TF32 and FP32-SIMT forms."""
    import torch
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    out = {}
    was = torch.backends.cuda.matmul.allow_tf32
    for name, tf32 in (("tf32_tflops", True), ("fp32_sgemm_tflops", False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2.0 * n ** 3 / best / 1e12
    torch.backends.cuda.matmul.allow_tf32 = was
    del a, b
    torch.cuda.empty_cache()
    return out


# -------------------------------------------------------------------------------------
# our arm
# -------------------------------------------------------------------------------------
def run_ours(args, W, ws, rank, local):
    import numpy as np
    import torch

    from paper_2308_07487_gb300 import asd, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    lat = W["lat"]
    N, F, T0, n_t, nb = lat.n_sites, W["F"], W["T0"], W["n_t"], W["n_bins"]
    q = W["q"]
    nq = 0 if q is None else len(q)
    nt_step = args.nt_per_step or W["nt_step"]
    nt_step = max(1, min(nt_step, n_t))
    n_blocks = (n_t + nt_step - 1) // nt_step
    K = 3 * T0
    flops_disp = 2.0 * N * N * K                     # algorithmic, per displacement
    mult = {"split_bf16": 3, "bf16": 1, "tf32": 1, "fp32": 1}[args.form]

    def block(k):
        """Displacements of step k: consecutive blocks of nt_step, wrapping around."""
        tb = (k % n_blocks) * nt_step
        return tb, min(n_t, tb + nt_step)

    # ---- inputs: thermalised start (off the timed region) ----
    sysm = asd.System(lat)
    spins0 = torch.from_numpy(synth.random_unit(N, 23083 + rank)[None]).to(dev)
    sysm.thermalize(spins0, W["T"], W["sweeps"], asd.ASD_METROPOLIS, cone=0.0, adapt=True,
                    seed=23083 + rank)
    traj = torch.empty((N, 1, F, 3), dtype=torch.float32, device=dev)
    plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, W["w"], nb, precision=args.form, q=q,
                                    cta_pair=args.cta_pair and args.form != "fp32")
    C_sum = torch.zeros((n_t, nb), dtype=torch.float64, device=dev)
    C = torch.zeros_like(C_sum)
    Sq_sum = torch.zeros((n_t, nq), dtype=torch.float64, device=dev) if nq else None
    Sq = torch.zeros_like(Sq_sum) if nq else None

    def new_event():
        return torch.cuda.Event(enable_timing=True)

    def step(k, kernel_events=None):
        """One pass of the hot path over displacement block k; kernel_events (start,
        end) bracket the contraction kernel on the stream it is launched on."""
        tb, te = block(k)
        sysm.ll_integrate(spins0, W["dt"], F, 1, traj, stream=stream)
        C_sum.zero_()
        if nq:
            Sq_sum.zero_()
        plan.prepare(traj, stream=stream)
        if kernel_events is not None:
            kernel_events[0].record(stream)
        plan.contract(C_sum, Sq_sum, stream=stream, t_range=(tb, te))
        if kernel_events is not None:
            kernel_events[1].record(stream)
        plan.normalize(C_sum, Sq_sum, C, Sq, stream=stream)
        return te - tb

    if args.ncu:
        step(0)
        asd.check(asd.sync_status(stream), "step")
        return

    for k in range(args.warmup):
        step(k)
    asd.check(asd.sync_status(stream), "warmup")

    ktimes, work = [], 0
    t_start, t_end = new_event(), new_event()
    barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            pair = (new_event(), new_event())
            nd = step(args.warmup + k, pair)
            ktimes.append((pair, nd))
            work += nd
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    asd.check(asd.sync_status(stream), "timed steps")
    t_total = t_start.elapsed_time(t_end) / 1e3
    t_total = allmax(ws, t_total)
    t_step = t_total / args.steps
    t_kernel = sum(a.elapsed_time(b) for (a, b), _ in ktimes) / 1e3
    clocks = clk.summary()
    value = flops_disp * work * ws / t_total / 1e12

    pk, pk_kind = peaks()
    extra_pk = measured_extra_peaks() if (not args.no_extras and rank == 0) else {}
    if args.form == "fp32":
        peak = extra_pk.get("fp32_sgemm_tflops")
        bound, punit, psrc = "alu", "TFLOP/s", "measured cuBLAS FP32 SGEMM (FFMA) in this run"
    elif args.form == "tf32":
        peak = extra_pk.get("tf32_tflops")
        bound, punit, psrc = "tensor", "TFLOP/s", "measured cuBLAS TF32 GEMM in this run"
    else:
        # a kernel timed inside a seconds-long step: the sustained BF16 figure
        peak = pk["bf16_tflops_sustained"]
        bound, punit, psrc = "tensor", "TFLOP/s", f"{pk_kind} bf16_tflops_sustained"
    achieved = flops_disp * work * mult / t_kernel / 1e12
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": punit,
            "frac": (achieved / peak) if peak else None, "traffic": None,
            "peak_source": psrc,
            "kernel": "pc_tc_kernel" if args.form != "fp32" else "simt_kernel",
            "flops_per_launch": flops_disp * nt_step * mult,
            "flops_note": "issued tensor flops of the contraction (x3 for split-BF16); the "
                          "phase weights are extra work and not counted",
            "algorithmic_tflops": flops_disp * work / t_kernel / 1e12,
            "kernel_ms": t_kernel / args.steps * 1e3}
    tfile = os.path.join(ROOT, "profiles", f"traffic_{args.form}_{W['name']}.txt")
    if os.path.exists(tfile):
        for line in open(tfile):
            if line.startswith("dram_bytes_per_launch:"):
                roof["traffic"] = float(line.split(":")[1])
    if extra_pk:
        roof["measured_peaks"] = extra_pk

    # per step: LL frame 0 + 4 RK4 stages per step, prep B + prep A copies (the FP32 form
    # prepares B only), the fused contraction, normalisation (the memsets are torch's)
    per_step = 1 + 4 * (F - 1) + (1 if args.form == "fp32" else 2) + 1 + 1
    out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": {"split_bf16": "bf16x3", "bf16": "bf16", "tf32": "tf32", "fp32": "f32"}[args.form],
           "data": "synthetic",
           "config": {"workload": W["name"], "N": N, "F": F, "T0": T0, "n_t": n_t,
                      "n_t_per_step": nt_step, "n_bins": nb, "bin_width": W["w"], "n_q": nq,
                      "K": K, "form": args.form, "parallelism": f"replicas x{ws}",
                      "cta_pair": bool(args.cta_pair and args.form != "fp32"),
                      "l2": "inputs larger than L2 (operand copies "
                            f"{plan.workspace_bytes() / 1e9:.1f} GB, trajectory "
                            f"{traj.numel() * 4 / 1e9:.2f} GB)"},
           "roofline": roof, "clocks": clocks,
           "gpu_launches": args.steps * per_step}

    # ---- extras (rank 0): precision forms, CPU oracle baseline + parity ----
    if not args.no_extras and rank == 0:
        tr_np = traj.cpu().numpy()
        # the oracle's sample: 4 rows per OpenMP thread, at the first and last displacement
        import oracle
        rows_o = (N // 2, min(N, N // 2 + oracle_rows(oracle.threads())))
        t_o = [0, n_t - 1]
        res, dt_o, fl_o = oracle_sample(W, tr_np, rows_o, t_o)
        out["cpu_baseline"] = {
            "value": fl_o / dt_o / 1e12, "unit": "TFLOP/s",
            "cores": min(oracle.threads(), rows_o[1] - rows_o[0]), "kind": "oracle",
            "sample": f"rows {rows_o[0]}..{rows_o[1]} x {N} columns x t {t_o}, K={K}, {nb} bins, "
                      f"{nq} q, {dt_o:.1f} s"}
        # every form: time on whole-N displacement blocks (FP32: an eighth of the rows,
        # scaled), errors on the oracle's rows
        forms = {}
        nt_f = min(2, n_t)
        for form in ("fp32", "tf32", "bf16", "split_bf16"):
            p2 = asd.CorrPlan.for_lattice(lat, F, T0, n_t, W["w"], nb, precision=form, q=q)
            c2 = torch.zeros((n_t, nb), dtype=torch.float64, device=dev)
            s2 = torch.zeros((n_t, nq), dtype=torch.float64, device=dev) if nq else None
            p2.prepare(traj, stream=stream)
            rows_t = (0, N // 8) if form == "fp32" else (0, N)
            scale = N / (rows_t[1] - rows_t[0])
            p2.contract(c2, s2, rows=rows_t, stream=stream, t_range=(0, 1))
            torch.cuda.synchronize()
            a, b = new_event(), new_event()
            a.record(stream)
            p2.contract(c2, s2, rows=rows_t, stream=stream, t_range=(0, nt_f))
            b.record(stream)
            torch.cuda.synchronize()
            dt = a.elapsed_time(b) / 1e3 * scale
            c2.zero_()
            if nq:
                s2.zero_()
            for t in t_o:
                p2.contract(c2, s2, rows=rows_o, stream=stream, t_range=(t, t + 1))
            asd.check(asd.sync_status(stream), f"form {form}")
            cs_o = c2.cpu().numpy()[t_o]
            rec = {"TFLOP/s": flops_disp * nt_f / dt / 1e12,
                   "sample": f"{nt_f} displacements" + (", rows 0..N/8 scaled" if form == "fp32"
                                                        else ""),
                   # the bar per bin on bins with >= 16 sampled pairs; every bin in units of
                   # the sum of |products| (the far bins of a row sample hold single pairs)
                   "max_bin_err": float(oracle.sampled_bin_error(cs_o, res).max()),
                   "max_bin_err_any_bin": float(oracle.bin_error(cs_o, res).max()),
                   "max_err_vs_sum_abs_products": float(oracle.rounding_ratio(cs_o, res).max())}
            if nq:
                rec["max_phase_err"] = float(oracle.phase_error(s2.cpu().numpy()[t_o], res).max())
            forms[form] = rec
            p2.close()
        out["forms"] = forms
        out["speedup_split_bf16_vs_fp32"] = forms["split_bf16"]["TFLOP/s"] / forms["fp32"]["TFLOP/s"]
        if extra_pk:
            out["fp32_form_frac_of_sgemm"] = forms["fp32"]["TFLOP/s"] / extra_pk["fp32_sgemm_tflops"]
        out["max_bin_err"] = forms[args.form]["max_bin_err"]
        out["max_err_vs_sum_abs_products"] = forms[args.form]["max_err_vs_sum_abs_products"]
        if nq:
            out["max_phase_err"] = forms[args.form]["max_phase_err"]
            # the phase sums through the separable transform route (all displacements)
            p3 = asd.CorrPlan.for_lattice(lat, F, T0, n_t, W["w"], 0, q=q)
            s3 = torch.zeros((n_t, nq), dtype=torch.float64, device=dev)
            p3.sq_separable(traj, s3, stream=stream)
            torch.cuda.synchronize()
            a, b = new_event(), new_event()
            a.record(stream)
            p3.sq_separable(traj, s3, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            s3.zero_()
            p3.sq_separable(traj, s3, stream=stream)
            asd.check(asd.sync_status(stream), "separable")
            # against the fused sums of the last timed step's displacements (all rows)
            tb, te = block(args.warmup + args.steps - 1)
            fs, ss = Sq_sum.cpu().numpy()[tb:te], s3.cpu().numpy()[tb:te]
            out["separable_phase"] = {
                "displacements": n_t, "ms": a.elapsed_time(b),
                "rel_diff_vs_fused": float(np.abs(ss - fs).max() / np.abs(fs).max())}
            p3.close()
            # the same kernel with bins only (what the phase epilogue costs)
            p4 = asd.CorrPlan.for_lattice(lat, F, T0, n_t, W["w"], nb, precision=args.form)
            c4 = torch.zeros((n_t, nb), dtype=torch.float64, device=dev)
            p4.prepare(traj, stream=stream)
            p4.contract(c4, None, stream=stream, t_range=(0, 1))
            torch.cuda.synchronize()
            a, b = new_event(), new_event()
            a.record(stream)
            p4.contract(c4, None, stream=stream, t_range=(0, nt_f))
            b.record(stream)
            torch.cuda.synchronize()
            asd.check(asd.sync_status(stream), "bins only")
            out["bins_only_TFLOP/s"] = flops_disp * nt_f / (a.elapsed_time(b) / 1e3) / 1e12
            p4.close()
        del tr_np

    if not args.no_extras:
        # e2e through the public API on every rank: pinned host spins -> device, full step,
        # C(b,t) and S(q,t) of the step's block -> host; the job's time is the slowest rank's
        h_in = torch.from_numpy(spins0.cpu().numpy()).pin_memory()
        h_c = torch.empty((n_t, nb), dtype=torch.float64).pin_memory()
        h_q = torch.empty((n_t, nq), dtype=torch.float64).pin_memory() if nq else None
        a = new_event()
        b = new_event()
        d2h = 0
        barrier(ws)
        torch.cuda.synchronize()
        with Clocks(local) as clk_e2e, torch.cuda.stream(stream):
            t0 = time.perf_counter()
            a.record(stream)
            work_e = 0
            for k in range(args.steps):
                spins0.copy_(h_in, non_blocking=True)
                tb, te = block(args.warmup + k)
                work_e += step(args.warmup + k)
                h_c[tb:te].copy_(C[tb:te], non_blocking=True)
                d2h += (te - tb) * nb * 8
                if nq:
                    h_q[tb:te].copy_(Sq[tb:te], non_blocking=True)
                    d2h += (te - tb) * nq * 8
            b.record(stream)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) / args.steps
        barrier(ws)
        te_s = allmax(ws, a.elapsed_time(b) / 1e3)
        wall = allmax(ws, wall)
        # (a separate run of the same steps: its SM clock under the power cap is recorded,
        # since it can differ from the clock of the device-timed run)
        out["e2e"] = {"value": flops_disp * work_e * ws / te_s / 1e12, "unit": "TFLOP/s",
                      "h2d_bytes_per_step": int(h_in.numel() * 4),
                      "d2h_bytes_per_step": int(d2h // args.steps),
                      "wall_s_per_step": wall, "clocks": clk_e2e.summary()}
    if rank == 0:
        print(json.dumps(out))
    plan.close()


# -------------------------------------------------------------------------------------
# other workloads (one JSON line each; the headline line is the glass64 workload)
# -------------------------------------------------------------------------------------
def _timed(fn, reps=1):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def run_ensemble(args):
    """96 independent 2D/3D periodic samples, N_s log-uniform in [1024, 40000], each with
    its own lattice, bins and plan; F = 320, T0 = 256, 64 displacements, split-BF16.
    One persistent launch over all problems (asd_pair_corr_batched), the same captured
    in a CUDA graph and replayed, and 96 separate launches."""
    import torch

    from paper_2308_07487_gb300 import asd, synth
    F, T0, n_t = 320, 256, 64
    sizes = synth.ensemble_sizes(96)
    plans, trajs, Cs, fl, lat_list = [], [], [], 0.0, []
    for k, (d, L) in enumerate(sizes):
        lat = synth.hypercubic(L, d, True, J=1.0)
        w = 1.0 if d == 2 else 0.5
        rmax = (d * (L // 2) ** 2) ** 0.5
        nb = int(rmax / w) + 1
        sysm = asd.System(lat)
        sp = torch.from_numpy(synth.random_unit(lat.n_sites, 23084 + k)[None]).cuda()
        sysm.thermalize(sp, 0.5 if d == 2 else 1.2, 200, asd.ASD_METROPOLIS, adapt=True,
                        seed=23084 + k)
        tr = torch.empty((lat.n_sites, 1, F, 3), dtype=torch.float32, device="cuda")
        sysm.ll_integrate(sp, 0.01, F, 1, tr)
        plans.append(asd.CorrPlan.for_lattice(lat, F, T0, n_t, w, nb, precision="split_bf16",
                                              tile_n=256))
        lat_list.append((lat, w, nb))
        trajs.append(tr)
        Cs.append(torch.zeros((n_t, nb), dtype=torch.float64, device="cuda"))
        fl += 2.0 * lat.n_sites ** 2 * 3 * T0 * n_t
    torch.cuda.synchronize()
    t_sep = _timed(lambda: [p.run(t, c) for p, t, c in zip(plans, trajs, Cs)])
    t_bat = _timed(lambda: asd.pair_corr_batched(plans, trajs, Cs))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        asd.pair_corr_batched(plans, trajs, Cs, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        asd.pair_corr_batched(plans, trajs, Cs, stream=s)
    t_graph = _timed(lambda: g.replay())
    asd.check(asd.sync_status(), "ensemble")
    # autotuned shared launch knobs (timed on 4 displacements of the whole batch)
    from paper_2308_07487_gb300 import tune
    probs = [(pl_lat, pl_w, pl_nb) for pl_lat, pl_w, pl_nb in lat_list]
    t0 = time.perf_counter()
    best = tune.Tuner().tune_batch(asd, probs, F, T0, trajs, n_t_sample=4,
                                   space={"tile_n": [128, 256], "epi_warps": [4, 8],
                                          "raster_m": [16, 32]})
    t_tune = time.perf_counter() - t0
    tplans = [asd.CorrPlan.for_lattice(pl_lat, F, T0, n_t, pl_w, pl_nb, precision="split_bf16",
                                       **best) for pl_lat, pl_w, pl_nb in lat_list]
    t_tuned = _timed(lambda: asd.pair_corr_batched(tplans, trajs, Cs))
    for p in tplans:
        p.close()
    print(json.dumps({
        "workload": "ensemble96_uneven", "metric": "fused pair-corr TFLOP/s (split-BF16)",
        "unit": "TFLOP/s", "n_samples": len(plans),
        "N_range": [min(p.N for p in plans), max(p.N for p in plans)],
        "total_sites": int(sum(p.N for p in plans)),
        "batched_one_launch": fl / t_bat / 1e12, "graph_replay": fl / t_graph / 1e12,
        "separate_launches": fl / t_sep / 1e12,
        "batched_autotuned": fl / t_tuned / 1e12, "autotuned_knobs": best,
        "autotune_s": t_tune,
        "ms": {"batched": t_bat * 1e3, "graph": t_graph * 1e3, "separate": t_sep * 1e3,
               "batched_autotuned": t_tuned * 1e3}}))
    for p in plans:
        p.close()


def run_learned(args):
    """128^2 periodic lattice, J = +1, T = 0.7: train the vMF proposal network on plain
    Metropolis configurations with the GPU kernels, sample 64 starts with the learned
    proposal and with plain Metropolis, integrate LL (F = 576) and correlate the 64 starts
    concatenated along K (T0 = 512, 64 displacements, K = 3 x 512 x 64)."""
    import math

    import numpy as np
    import torch

    from paper_2308_07487_gb300 import asd, synth
    L, T, S = 128, 0.7, 64
    lat = synth.hypercubic(L, 2, True, J=1.0)
    N = lat.n_sites
    sysm = asd.System(lat)
    sp = torch.from_numpy(synth.random_unit(S * N, 23085).reshape(S, N, 3)).cuda()
    sysm.thermalize(sp, T, 1000, asd.ASD_METROPOLIS, adapt=True, seed=23085)
    xs, ys = [], []
    nconf = 10000 // S + 1                       # ~10^4 training configurations
    t0 = time.perf_counter()
    for k in range(nconf):
        sysm.thermalize(sp, T, 2, asd.ASD_METROPOLIS, adapt=True, seed=23085, counter=1000 + 2 * k)
        if k % 8 == 0:
            x = torch.empty((S * N, 12), device="cuda")
            y = torch.empty((S * N, 3), device="cuda")
            sysm.gather(sp, x, y)
            xs.append(x)
            ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = asd.Mlp(12, seed=5, depth=args.mlp_depth)
    gen = torch.Generator(device="cuda").manual_seed(0)
    B, steps = 16384, 1500
    t0 = time.perf_counter()
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (B,), device="cuda", generator=gen)
        net.grad.zero_()
        net.loss.zero_()
        net.loss_grad(X[idx].contiguous(), Y[idx].contiguous())
        net.adam(lr=3e-3 if it < 1000 else 1e-3, scale=1.0 / B)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    net.grad.zero_()
    net.loss.zero_()
    net.loss_grad(X[:262144].contiguous(), Y[:262144].contiguous())
    nll = net.loss.item() / 262144

    def chain(prop, kw):
        s2 = sp.clone()
        sysm.thermalize(s2, T, 200, prop, seed=7, **kw)
        es, ms, acc, pr = [], [], 0, 0
        e_smp, m_smp = [], []
        for k in range(100):
            st = sysm.thermalize(s2, T, 2, prop, seed=7, counter=200 + 2 * k, stats=True, **kw)
            pr += st[0]
            acc += st[1]
            y = s2.double()
            e = torch.zeros(S, dtype=torch.float64, device="cuda")
            for a in range(lat.nbr.shape[1]):
                e += (y * y[:, torch.from_numpy(lat.nbr[:, a]).long().cuda()]).sum(dim=(1, 2))
            e = (e / 2 / N).cpu().numpy()              # per sample, energy per site (J = 1)
            m = y.mean(1).norm(dim=1).cpu().numpy()    # per sample |M| / N
            e_smp.append(e)
            m_smp.append(m)
            es.append(float(e.mean()))
            ms.append(float(m.mean()))
        hist_e[prop] = np.concatenate(e_smp)
        hist_m[prop] = np.concatenate(m_smp)
        es = np.array(es)
        # integrated autocorrelation time of the energy per site, in units of the 2-sweep
        # measurement interval: normalised autocorrelation of each chain's series, averaged
        # over the chains, summed up to its first non-positive lag
        E = np.stack(e_smp, 1)                                   # [chains][measurements]
        X = E - E.mean(axis=1, keepdims=True)
        var = (X * X).mean()
        n_meas = X.shape[1]
        rho = [float((X[:, :n_meas - k] * X[:, k:]).mean() / var) for k in range(1, 30)]
        tau = 0.5
        for r in rho:
            if r <= 0:
                break
            tau += r
        return s2, {"acceptance": acc / pr, "energy_per_site": float(es.mean()),
                    "energy_sem": float(es.std() / math.sqrt(len(es))), "tau_int_energy": tau,
                    "magnetisation": float(np.mean(ms))}
    hist_e, hist_m = {}, {}
    s_learn, st_learn = chain(asd.ASD_LEARNED, {"net": net})
    s_metro, st_metro = chain(asd.ASD_METROPOLIS, {"cone": 0.0})
    _, st_heat = chain(asd.ASD_HEATBATH, {})

    def ks(a, b):
        """Two-sample Kolmogorov-Smirnov statistic (largest gap between the ECDFs)."""
        z = np.sort(np.concatenate([a, b]))
        return float(np.abs(np.searchsorted(np.sort(a), z, "right") / len(a)
                            - np.searchsorted(np.sort(b), z, "right") / len(b)).max())

    def hist(x, lo, hi):
        h, _ = np.histogram(x, bins=20, range=(lo, hi))
        return (h / len(x)).round(4).tolist()
    elo = min(v.min() for v in hist_e.values())
    ehi = max(v.max() for v in hist_e.values())
    mhi = max(v.max() for v in hist_m.values())
    L_, M_, H_ = asd.ASD_LEARNED, asd.ASD_METROPOLIS, asd.ASD_HEATBATH
    histograms = {
        "samples_per_method": int(len(hist_e[L_])),
        "ks_energy": {"learned_vs_heatbath": ks(hist_e[L_], hist_e[H_]),
                      "metropolis_vs_heatbath": ks(hist_e[M_], hist_e[H_])},
        "ks_magnetisation": {"learned_vs_heatbath": ks(hist_m[L_], hist_m[H_]),
                             "metropolis_vs_heatbath": ks(hist_m[M_], hist_m[H_])},
        "energy_range": [float(elo), float(ehi)], "magnetisation_range": [0.0, float(mhi)],
        "energy_hist": {k: hist(hist_e[v], elo, ehi) for k, v in
                        (("learned", L_), ("metropolis", M_), ("heatbath", H_))},
        "magnetisation_hist": {k: hist(hist_m[v], 0.0, mhi) for k, v in
                               (("learned", L_), ("metropolis", M_), ("heatbath", H_))}}
    F, T0, n_t = 576, 512, 64
    res = {}
    for name, starts in (("learned", s_learn), ("metropolis", s_metro)):
        tr = torch.empty((N, S, F, 3), dtype=torch.float32, device="cuda")
        sysm.ll_integrate(starts, 0.01, F, 1, tr)
        plan = asd.CorrPlan.for_lattice(lat, F, T0, n_t, 1.0, 91, precision="split_bf16", S=S)
        C = torch.zeros((n_t, 91), dtype=torch.float64, device="cuda")
        plan.prepare(tr)
        dt = _timed(lambda: plan.contract(C))
        C.zero_()
        plan.contract(C)
        Cn = torch.zeros_like(C)
        plan.normalize(C, None, Cn, None)
        torch.cuda.synchronize()
        if name == "learned":
            # per-bin error against the FP64 oracle on 4 rows x all columns
            import oracle
            rows = (5000, 5004)
            Cr = torch.zeros_like(C)
            plan.contract(Cr, rows=rows)
            tr_h = tr.cpu().numpy()
            ref = oracle.pair_corr(tr_h, T0, [0, n_t - 1], oracle.Geometry.of_lattice(lat),
                                   1.0, 91, rows=rows)
            err_rows = float(oracle.bin_error(Cr.cpu().numpy()[[0, n_t - 1]], ref).max())
            del tr_h
        fl = 2.0 * N * N * 3 * T0 * S * n_t
        res[name] = {"C": Cn.cpu().numpy(), "TFLOP/s": fl / dt / 1e12, "ms": dt * 1e3}
        plan.close()
    dC = np.abs(res["learned"]["C"] - res["metropolis"]["C"])[:, :40].max()
    print(json.dumps({
        "workload": "sq128_learned_proposal", "T": T, "starts": S, "mlp_depth": args.mlp_depth,
        "training": {"pairs": int(X.shape[0]), "steps": steps, "batch": B,
                     "data_s": t_data, "train_s": t_train, "nll_per_site": nll,
                     "nll_uniform": math.log(4 * math.pi)},
        "chains": {"learned": st_learn, "metropolis": st_metro, "heatbath": st_heat},
        "histograms": histograms,
        "corr_TFLOP/s": {k: v["TFLOP/s"] for k, v in res.items()},
        "corr_ms": {k: v["ms"] for k, v in res.items()},
        "max_abs_C_diff_learned_vs_metropolis_r<40": float(dC),
        "corr_max_bin_err_rows_5000_5004": err_rows}))


def run_kernels(args):
    """One small launch of every library kernel besides the fused contraction, for the
    per-kernel ncu summaries (capture with -k regex:<kernel> -c <n>): the FP32 SIMT form,
    operand preparation, pair counts and normalisation on a 32^3 jittered glass
    (N = 32768, F = 640, T0 = 512, 256 bins, 64 q; operands ~1 GB, larger than L2); the
    separable phase route (transform + time correlation) and S(q, omega) on the same glass;
    Monte Carlo sweeps (Metropolis, heat-bath, learned), LL RK4 stages and the network's
    initialiser, gather, loss/gradient, Adam and BF16-copy kernels on a 256^2 lattice (16
    samples, 10^6 sites).  Prints one JSON line of CUDA-event times per call."""
    import torch

    from paper_2308_07487_gb300 import asd, synth
    ev = {}

    def timed(name, fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        asd.check(asd.sync_status(), name)
        ev[name] = a.elapsed_time(b)

    glass = synth.hypercubic(32, 3, False, pm_j=True, p=0.5, seed=7, block=(4, 4, 8), jitter=0.1)
    q = synth.q_vectors_glass()
    N, F, T0, nt = glass.n_sites, 640, 512, 128
    tr = torch.from_numpy(synth.traj_precess(N, F, seed=5)).cuda()
    plan = asd.CorrPlan.for_lattice(glass, F, T0, nt, 0.5, 256, precision="fp32", q=q)
    C = torch.zeros((nt, 256), dtype=torch.float64, device="cuda")
    Sq = torch.zeros((nt, 64), dtype=torch.float64, device="cuda")
    timed("prepare_fp32", lambda: plan.prepare(tr))
    timed("simt_contract_rows4096_t1", lambda: plan.contract(C, Sq, rows=(0, 4096), t_range=(0, 1)))
    timed("normalize", lambda: plan.normalize(C, Sq, C, Sq))
    timed("separable_128_displacements", lambda: plan.sq_separable(tr, Sq))
    omega = torch.linspace(0.0, 20.0, 512, dtype=torch.float64, device="cuda")
    Sqw = torch.zeros((512, 64), dtype=torch.float64, device="cuda")
    timed("sq_omega_512", lambda: asd.sq_omega(Sq, 0.01, omega, Sqw))
    plan.close()
    plan2 = asd.CorrPlan.for_lattice(glass, F, T0, nt, 0.5, 256, precision="split_bf16", q=q)
    timed("prepare_split_bf16", lambda: plan2.prepare(tr))
    plan2.close()
    del tr
    torch.cuda.empty_cache()
    lat = synth.hypercubic(256, 2, True, J=1.0)
    S = 16
    sysm = asd.System(lat)
    sp = torch.from_numpy(synth.random_unit(S * lat.n_sites, 3).reshape(S, lat.n_sites, 3)).cuda()
    net = asd.Mlp(12, seed=1)
    timed("mc_metropolis_sweep", lambda: sysm.thermalize(sp, 0.7, 1, asd.ASD_METROPOLIS, seed=1))
    timed("mc_heatbath_sweep", lambda: sysm.thermalize(sp, 0.7, 1, asd.ASD_HEATBATH, seed=1))
    timed("mc_learned_sweep", lambda: sysm.thermalize(sp, 0.7, 1, asd.ASD_LEARNED, net=net, seed=1))
    trl = torch.empty((lat.n_sites, S, 2, 3), dtype=torch.float32, device="cuda")
    timed("ll_one_rk4_step", lambda: sysm.ll_integrate(sp, 0.01, 2, 1, trl))
    x = torch.empty((S * lat.n_sites, 12), device="cuda")
    y = torch.empty((S * lat.n_sites, 3), device="cuda")
    timed("mlp_gather", lambda: sysm.gather(sp, x, y))
    timed("mlp_loss_grad_262144", lambda: net.loss_grad(x[:262144], y[:262144]))
    timed("mlp_adam", lambda: net.adam(lr=1e-3, scale=1.0 / 262144))
    timed("mlp_init", lambda: asd.Mlp(12, seed=2))
    timed("mlp_weights_bf16", lambda: net._refresh_bf16())
    print(json.dumps({"workload": "kernels", "ms": ev}))


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.workload in ("ensemble", "learned", "kernels"):
        if rank == 0:
            {"ensemble": run_ensemble, "learned": run_learned,
             "kernels": run_kernels}[args.workload](args)
        return
    W = workload(args.workload, args.small, args.medium)
    if args.impl == "reference":
        run_reference(args, W, ws, rank)
    else:
        run_ours(args, W, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
