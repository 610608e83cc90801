#!/usr/bin/env python3
"""Benchmark of the Wiener-reconstruction hot path on one GB300 (or N replicas).

One step = the whole hot path over one synthetic 512^3 catalogue held in HBM:
supersampled TSC gridding (1024^3 fine grid, ideal low-pass) -> window/noise -> Wiener solve
to relative residual 1e-6 (mixed precision: FP32-FFT inner CG preconditioned on the coarse
Fourier modes |k| <= K, FP64 refinement).  The same step without the coarse space and the FP64
form are timed beside it.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wf|reference] [--workload c3|c2|c1]
                  [--deflate K]   (coarse radius of the mixed solves; -1: by grid size, 0: none)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "512^3 Wiener-CG solves/s to 1e-6 residual, mixed vs FP64; HBM GB/s; p50/p99"
WORKLOADS = {
    "c3": "512^3 grid, 500 Mpc/h box, ~5e5 log-normal galaxies (seed 1003), LCDM P(k) sigma8=0.8, "
          "gamma-law radial selection (peak 150 Mpc/h), 30-deg cone with 5% holes; TSC, supersampling 2 "
          "(1024^3 fine grid); CG to 1e-6",
    "c2": "256^3 grid, 500 Mpc/h box, 1.5e5 log-normal galaxies (seed 1002), same P(k)/selection; TSC s=2; CG 1e-6",
    "c1": "64^3 grid, 200 Mpc/h box, 2e4 log-normal galaxies (seed 1001), P=A k^-1.5; CIC s=2; CG 1e-8",
}
# DRAM traffic of the dominant kernel per launch from one ncu capture, valid while the kernel
# sources hash to `src`; scaled from the captured size by the units processed (bytes ~ N^3).
NCU_TRAFFIC = {
    # profiles/cg_kernels_f32_512_dram.md: one-pass capture of the launches of a deflated 512^3
    # iteration: x pass 1 1684.4 + 1555.2 MB; y pass (mean of the +1 and -1 launches) 536.9 + 472.1 MB
    ("cg_xinv", 512): {"bytes": 3239.6e6, "src": "f795d92c5a0ea8e0"},
    ("ypass", 512): {"bytes": 1009.0e6, "src": "f795d92c5a0ea8e0"},
}


def kernel_src_hash():
    h = hashlib.sha256()
    for f in ("wf_fft.cuh", "wf_spectral.cuh", "wf_common.cuh"):
        with open(os.path.join(ROOT, "paper_0906_3978_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        # nvidia-smi numbers physical GPUs and ignores CUDA_VISIBLE_DEVICES: select the GPU this
        # process runs on by its UUID instead of the CUDA ordinal
        self.index = index
        self.uuid = gpu_uuid(index)
        self.p = None

    def __enter__(self):
        try:
            sel = self.uuid if self.uuid else str(self.index)
            self.p = subprocess.Popen(["nvidia-smi", "-i", sel, "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "gpu_uuid": self.uuid}


def gpu_uuid(index):
    """'GPU-xxxxxxxx-...' of CUDA device `index` (nvidia-smi's form), or None without torch/CUDA."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(index).uuid)
    except Exception:
        return None
    return u if u.startswith("GPU-") else "GPU-" + u


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("WF_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier_max(ws, t):
    """Maximum of t over the ranks (the slowest rank's time)."""
    if ws == 1:
        return t
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    v = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------
# CPU oracle baseline: bounded sample of the same workload on the host cores
# ------------------------------------------------------------------------------------------
def oracle_sample(pr, iters, deadline_s=40.0, single_thread=True):
    """Time the oracle on a bounded sample of the workload and scale it to solves/s:
    full-size assignment and window, one textbook-CG matvec at full size, the ideal low-pass
    counted as 5 matvecs (a 1024^3 and a 512^3 complex transform), and `iters` iterations."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    fine = oracle.assign(pr.pos, pr.n, pr.box, pr.scheme, 2)
    del fine
    t_assign = time.perf_counter() - t0
    t0 = time.perf_counter()
    w = oracle.window(pr.sel, pr.n, pr.box)
    t_window = time.perf_counter() - t0
    tab = oracle.sinv_table(pr.n, pr.box, pr.pk_k, pr.pk_p)
    p = np.ones_like(w)
    t0 = time.perf_counter()
    oracle.matvec(tab, 0.05, w, p)
    t_mv = time.perf_counter() - t0
    t_solve = t_assign + t_window + (iters + 5) * t_mv
    sample = ("oracle (plain C, FP64, %d OpenMP threads) at %d^3: assignment of all %d galaxies onto the 2x fine "
              "grid (%.2f s), window (%.2f s), one CG matvec (%.2f s); solve = assignment + window + (%d CG "
              "iterations as the GPU FP64 solve needed + 5 for the low-pass) x matvec"
              % (oracle.threads(), pr.n, pr.n_gal, t_assign, t_window, t_mv, iters))
    if not single_thread:
        return 1.0 / t_solve, oracle.threads(), sample, t_solve, None
    # one thread: a 256^3 matvec, scaled to 512^3 by V log V (x 9)
    nt = oracle.threads()
    n1 = pr.n // 2
    tab1 = oracle.sinv_table(n1, pr.box, pr.pk_k, pr.pk_p)
    w1 = np.ones((n1, n1, n1))
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.matvec(tab1, 0.05, w1, w1)
        t_mv1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(nt)
    scale = 8.0 * math.log2(pr.n ** 3) / math.log2(n1 ** 3)
    single = {"matvec_s_at_half_n": t_mv1, "matvec_s_extrapolated": t_mv1 * scale,
              "threads_speedup_on_matvec": t_mv1 * scale / t_mv,
              "note": "1 OpenMP thread, one %d^3 matvec scaled by V log V to %d^3" % (n1, pr.n)}
    return 1.0 / t_solve, oracle.threads(), sample, t_solve, single


def fp64_kernels(ctx, prof, n):
    """The FP64-ALU-bound passes of the step (the three passes of the ideal low-pass and the passes of
    the FP64 residual) against the device's FP64 rate measured here (wf_fp64_rate) and the nominal
    1.25 TFLOP/s.  Algorithmic flops:
    2.5 L log2 L per real transform of length L; each pass line takes a real transform of length 2n
    and an inverse of length n; the z pass has (2n)^2 lines, the y pass 2n n, the x pass n n.  The z
    pass skips the rows no galaxy reaches (their output is zero), so its figure counts flops it did
    not need to do."""
    peak = ctx.fp64_rate()
    f_line = 2.5 * 2 * n * math.log2(2 * n) + 2.5 * n * math.log2(n)
    lines = {"lowpass_z": (2 * n) ** 2, "lowpass_y": 2 * n * n, "lowpass_x": n * n}
    # the FP64 residual's passes (FP64 storage and arithmetic): per launch, the y pass takes n n/2
    # complex transforms of length n (5 n log2 n each), the x pass with the Fourier table two of them
    # (forward and inverse), the z passes n^2 real transforms of length n (2.5 n log2 n each)
    cplx = 5.0 * n * math.log2(n)
    flops = {"ypass_f64": n * n / 2 * cplx, "xmul_f64": 2 * n * n / 2 * cplx,
             "zfwd_f64": n * n * cplx / 2, "zinv_f64": n * n * cplx / 2}
    out = []
    for c in prof["classes"]:
        if (c["name"] in lines or c["name"] in flops) and c["launches"] > 0:
            fl = lines[c["name"]] * f_line if c["name"] in lines else flops[c["name"]]
            rate = fl / (c["ms"] / c["launches"] / 1000.0)
            out.append({"kernel": c["name"], "bound": "alu", "gflop_per_launch": fl / 1e9,
                        "ms_per_launch": c["ms"] / c["launches"], "achieved_tflops": rate / 1e12,
                        "frac_of_measured": rate / peak, "frac_of_nominal": rate / 1.25e12})
    return {"peak_measured_tflops": peak / 1e12, "peak_nominal_tflops": 1.25,
            "peak_kind": "measured: wf_fp64_rate (FMA chains filling every SM, CUDA events)", "kernels": out}


def config_of(args, pr, ws):
    """The workload description both arms print (identical keys and values)."""
    return {"workload": WORKLOADS[args.workload], "n": pr.n, "n_gal": pr.n_gal,
            "l2": "inputs larger than L2 (fine grid 8.6 GB, spectra 0.5-1.1 GB at 512^3)",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def oracle_full_solve(name, threads):
    """Seconds of one whole oracle reconstruction of workload `name` (assignment, low-pass, window,
    noise, textbook CG to the workload's tolerance) on `threads` OpenMP threads, and its CG
    iterations."""
    import oracle
    import synth
    pr = synth.problem(name)
    nt = oracle.threads()
    oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        fine = oracle.assign(pr.pos, pr.n, pr.box, pr.scheme, 2)
        nobs = oracle.lowpass(fine, pr.n, 2)
        del fine
        w = oracle.window(pr.sel, pr.n, pr.box)
        d, b, nbar = oracle.build_noise(nobs, w, pr.n_gal)
        tab = oracle.sinv_table(pr.n, pr.box, pr.pk_k, pr.pk_p)
        x, it, rel = oracle.cg(tab, nbar, w, b, tol=pr.tol, max_iter=100000)
        return time.perf_counter() - t0, it, rel
    finally:
        oracle.set_threads(nt)


def reference_arm(args):
    ws, rank, _ = dist_init()
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    pr = synth.problem(args.workload)
    iters = REF_ITERS.get(args.workload, 200)
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, sample, t, _ = oracle_sample(pr, iters, single_thread=False)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, pr, args.gpus),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "extrapolated": True, "iterations_used": iters,
                             "iterations_source": ITERS_SOURCE},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# GPU FP64-solve iteration counts on each workload, used by the reference arm (which runs without
# a GPU) to scale its per-iteration time to a solve; the GPU arm uses the count it measures.
REF_ITERS = {"c3": 297, "c2": 150, "c1": 60}
ITERS_SOURCE = ("the GPU FP64 solve's CG iterations on this workload as bench.py's GPU arm measured them "
                "(512^3: 297); the GPU arm's own cpu_baseline uses the count of its run")


def cpu_model():
    """The host CPU's model name (/proc/cpuinfo, else lscpu), or the machine type."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def gpu_arm(args):
    ws, rank, local = dist_init()
    import numpy as np
    import torch
    import paper_0906_3978_gb300 as wf
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wf.build()
    pr = synth.problem(args.workload)
    ctx = wf.Context(local)
    st = torch.cuda.Stream(device=dev)
    pos = torch.from_numpy(pr.pos).to(dev)
    n, box = pr.n, pr.box
    tol = pr.tol
    # launch variants of the spectral passes timed once for this size (outside any timed region)
    tuning = {"mixed": ctx.autotune(n, wf.MIXED), "fp64": ctx.autotune(n, wf.FP64)}

    defl = args.deflate

    def step(prec, s_out=None, pos_d=pos, deflate=defl):
        with torch.cuda.stream(st):
            nobs = ctx.grid_assign(pos_d, n, box, pr.scheme, 2, stream=st)
            w, d, b, nbar = ctx.build_noise(pr.sel, nobs, pr.n_gal, box, stream=st, want_d=False)
            s, info = ctx.solve(w, nbar, b, box, pr.pk_k, pr.pk_p, tol=tol, max_iter=20000, prec=prec,
                                s_out=s_out, stream=st, deflate=deflate if prec == wf.MIXED else 0)
        return s, info

    def timed(prec, k, w_, profile=False, deflate=defl):
        for _ in range(w_):
            step(prec, deflate=deflate)
        torch.cuda.synchronize()
        barrier(ws)
        ctx.profile(profile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        infos = []
        for _ in range(k):
            s, info = step(prec, deflate=deflate)
            infos.append(info.as_dict())
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return ms, infos, s

    # ---- headline: mixed precision as a user runs it (CG blocks replayed as CUDA graphs); the
    # library counts every launch, graph members included
    with Clocks(local) as clk:
        ms_mixed, infos_mixed, s_mixed = timed(wf.MIXED, args.steps, args.warmup, profile=False)
    launches_timed = read_profile(ctx)["launches"]
    ms_mixed = barrier_max(ws, ms_mixed)
    # ---- the same steps again with a CUDA-event pair around every launch on its stream (direct
    # launches instead of graphs): the per-kernel durations behind the roofline
    timed(wf.MIXED, args.steps, 0, profile=True)
    prof = read_profile(ctx)
    # ---- the mixed step without the coarse space, and the FP64 form of the same step
    ctx.profile(False)
    if defl != 0:
        ms_plain, infos_plain, s_plain = timed(wf.MIXED, max(1, args.steps // 3), 1, deflate=0)
        ms_plain = barrier_max(ws, ms_plain)
        del s_plain
    ms_fp64, infos_fp64, s_fp64 = timed(wf.FP64, max(1, args.steps // 3), 1)
    ms_fp64 = barrier_max(ws, ms_fp64)
    ctx.profile(False)
    diff = float(torch.linalg.norm(s_mixed - s_fp64) / torch.linalg.norm(s_fp64))
    # error of each result against the solution converged to 1e-10 (FP64 refinement)
    nobs_r = ctx.grid_assign(pos, n, box, pr.scheme, 2)
    w_r, d_r, b_r, nbar_r = ctx.build_noise(pr.sel, nobs_r, pr.n_gal, box, want_d=False)
    s_ref, info_ref = ctx.solve(w_r, nbar_r, b_r, box, pr.pk_k, pr.pk_p, tol=1e-10, max_iter=20000, prec=wf.MIXED)
    nref = torch.linalg.norm(s_ref)
    err_mixed = float(torch.linalg.norm(s_mixed - s_ref) / nref)
    err_fp64 = float(torch.linalg.norm(s_fp64 - s_ref) / nref)
    del s_ref, nobs_r
    # ---- e2e through the C ABI with host buffers (positions in, solution out)
    # Each step copies its positions in and its solution out; the solution of step i goes to the
    # host on a copy stream while step i + 1 computes (two device and two host buffers), and the
    # timed region ends when the last copy has landed.
    pos_h = torch.from_numpy(pr.pos).pin_memory()
    s_h = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(2)]
    s_dev = [torch.empty((n, n, n), dtype=torch.float64, device=dev) for _ in range(2)]
    cp = torch.cuda.Stream(device=dev)
    landed = [None, None]
    step(wf.MIXED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        j = i % 2
        if landed[j] is not None:
            landed[j].synchronize()  # buffer j's previous copy is on the host before reuse
        with torch.cuda.stream(st):
            pos_d = pos_h.to(dev, non_blocking=True)
        step(wf.MIXED, s_out=s_dev[j], pos_d=pos_d)
        solved = torch.cuda.Event()
        solved.record(st)
        cp.wait_event(solved)
        with torch.cuda.stream(cp):
            s_h[j].copy_(s_dev[j], non_blocking=True)
        landed[j] = torch.cuda.Event()
        landed[j].record(cp)
    for e in landed:
        if e is not None:
            e.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = barrier_max(ws, e2e_s)

    extra = {}
    if not args.no_forms:
        extra["postproc"] = bench_postproc(ctx, pr, s_mixed, s_fp64, w_r, b_r, nbar_r, defl)
    del b_r
    if not args.no_forms:
        extra["batch"] = bench_batch(ctx, dev, defl)
        extra["serving"] = bench_serving(ctx, dev, defl)
        extra["jackknife"] = bench_jackknife(ctx, dev, defl)
    if rank != 0:
        return 0
    k = args.steps
    value = ws * k / (ms_mixed / 1000.0)
    peak, peak_kind = peaks()
    dom = max((c for c in prof["classes"] if c["bytes"] > 0), key=lambda c: c["ms"])
    achieved = dom["bytes"] / dom["launches"] / (dom["ms"] / dom["launches"] / 1000.0) / 1e9
    tr = NCU_TRAFFIC.get((dom["name"], n))
    traffic = tr["bytes"] if tr and tr.get("src") == kernel_src_hash() else None
    it_fp64 = infos_fp64[-1]["iters"]
    cpu_v, cores, sample, _, single = oracle_sample(pr, it_fp64)
    # whole oracle reconstructions of the 64^3 workload (seconds each), on all and on one thread
    import oracle
    t_all, it_c1, _ = oracle_full_solve("c1", oracle.threads())
    t_one, _, _ = oracle_full_solve("c1", 1)
    full = {"c1": {"workload": WORKLOADS["c1"], "cg_iters": it_c1, "threads": oracle.threads(),
                   "s": round(t_all, 3), "s_1_thread": round(t_one, 3), "solves_per_s": 1.0 / t_all,
                   "solves_per_s_1_thread": 1.0 / t_one},
            "c2": "bench.py --cpu-full (minutes of host time)"}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": k, "warmup": args.warmup,
        "ms_per_step": ms_mixed / k, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 FFT/CG inner, f64 dots+refinement", "data": "synthetic",
        "config": config_of(args, pr, ws),
        "mixed": {"iters": infos_mixed[-1]["iters"], "outer": infos_mixed[-1]["outer_iters"],
                  "rel_residual": infos_mixed[-1]["rel_residual"], "rel_l2_vs_fp64_solve": diff,
                  "rel_l2_vs_converged": err_mixed, "deflate": deflate_of(defl, n),
                  "coarse_space": "inner CG preconditioned on the Fourier modes |k| <= deflate (grid units), "
                                  "two-level A-DEF2 form; 0 = none"},
        "mixed_no_coarse_space": None if defl == 0 else {
            "value": ws * max(1, k // 3) / (ms_plain / 1000.0), "ms_per_step": ms_plain / max(1, k // 3),
            "iters": infos_plain[-1]["iters"], "rel_residual": infos_plain[-1]["rel_residual"]},
        "fp64": {"value": ws * max(1, k // 3) / (ms_fp64 / 1000.0), "ms_per_step": ms_fp64 / max(1, k // 3),
                 "iters": it_fp64, "rel_residual": infos_fp64[-1]["rel_residual"], "rel_l2_vs_converged": err_fp64},
        "converged_reference": "the same step's system solved to relative residual 1e-10 (mixed with FP64 "
                               "refinement; residual %.1e)" % info_ref.rel_residual,
        "roofline": {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peak,
                     "timing": "CUDA events around each launch on its stream, in a repeat of the timed steps",
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                     "avg_launch_ms": dom["ms"] / dom["launches"]},
        "kernels": [{k2: (round(v, 4) if isinstance(v, float) else v) for k2, v in c.items()}
                    for c in sorted(prof["classes"], key=lambda c: -c["ms"])[:10]],
        "fp64_kernels": fp64_kernels(ctx, prof, n),
        "tuning": {prec: {p["pass"]: {"chosen": p["chosen"],
                                      "ms": {v["name"]: round(v["ms"], 4) for v in p["variants"]}}
                          for p in rep} for prec, rep in tuning.items()},
        "cpu_baseline": {"value": cpu_v, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "extrapolated": True, "iterations_used": it_fp64,
                         "iterations_source": "this run's GPU FP64 solve", "cpu": cpu_model(),
                         "single_thread": single, "full_solves": full},
        "e2e": {"value": ws * k / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(pr.pos.nbytes),
                "d2h_bytes_per_step": int(n ** 3 * 8),
                "note": "pinned host buffers; each solution's copy to the host overlaps the next step"},
        "gpu_launches": launches_timed,
        "clocks": clk.summary(),
    }
    line.update(extra)
    print(json.dumps(line))
    ctx.close()
    return 0


# ------------------------------------------------------------------------------------------
# Batched form: 96 mocks of uneven size in one wf_solve_batch call
# ------------------------------------------------------------------------------------------
def batch_mocks(count=96, seed=2000):
    """Seeded mocks of the batched workload: N from {64, 96, 128, 192}, L = 1.953 N Mpc/h,
    1e4-1e5 galaxies (log-uniform), LCDM prior, SDSS-like selection with per-mock holes."""
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    k, p = synth.lcdm_table()
    out = []
    for i in range(count):
        n = int(rng.choice([64, 96, 128, 192]))
        box = 1.953 * n
        ng = float(np.exp(rng.uniform(np.log(1e4), np.log(1e5))))
        sel = synth.selection_sdss_like(box, seed + i)
        pos = synth._cached_catalogue("batch_n%d_s%d_g%d" % (n, seed + i, int(ng)),
                                      lambda: synth.lognormal_catalogue(n, box, k, p, sel, ng, seed + i))
        out.append((n, box, sel, pos, k, p))
    return out


def bench_postproc(ctx, pr, s_rec, s_ref, w, b, nbar, defl=0):
    """Sec. 4.1 / 5.5 evaluation of the 512^3 reconstruction: Gaussian smoothing at r_S = 10, 20,
    30 Mpc/h (FP64 transforms, FP64-ALU-bound), the quality measures of the mixed solution
    against the FP64 one, and the density statistics of the r_S = 10 field in the paper's radial
    shells and observed / unobserved regions (1 + delta bins of 0.03 from -1); also the solve with
    Z and B inside R and the projection of a sky map into the 3D mask."""
    import numpy as np
    import torch
    import paper_0906_3978_gb300 as wf
    n, box = pr.n, pr.box

    def timed(f, reps=3):
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    out = {"workload": "the 512^3 mixed-precision solution s (as delta), its FP64 counterpart as the "
                       "reference; smoothing radii 10/20/30 Mpc/h; shells [0,200), [200,400), [400,inf), "
                       "[0,600) Mpc/h from the observer; 200 bins of 0.03 in 1 + delta from -1; the "
                       "inverse-weighting grid of the same catalogue"}
    sm = torch.empty_like(s_rec)
    for rs in (10.0, 20.0, 30.0):
        ms, _ = timed(lambda: ctx.smooth(s_rec, box, rs, out=sm))
        out["smooth_r%d_ms" % int(rs)] = ms
    ms, q = timed(lambda: ctx.compare(s_rec, s_ref))
    out["compare"] = {"ms": ms, "gbs": 16.0 * n ** 3 / (ms * 1e6), **q}
    pos = torch.from_numpy(pr.pos).to(s_rec.device)
    ms, _ = timed(lambda: ctx.grid_assign_weighted(pos, ctx.selection_eval(pr.sel, pos, reciprocal=True), n, box,
                                                   pr.scheme, 2))
    out["inverse_weighting_ms"] = ms  # masses 1 / w at the galaxies, 1024^3 fine grid, low-pass
    # the variant with Z and B inside R (Sec. 3.3.2): bias 1, Kaiser beta = 0.24^0.6, sigma_v = 5 Mpc/h
    # (500 km/s), mixed precision to 1e-6; one solve, as the headline's solve is timed
    beta = 0.24 ** 0.6
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    s_m, info = ctx.solve_response(w, nbar, b, box, pr.pk_k, pr.pk_p, 1.0, beta, 5.0, tol=1e-6, max_iter=20000,
                                   prec=wf.MIXED, deflate=defl)
    e1.record()
    torch.cuda.synchronize()
    out["response_solve"] = {"ms": e0.elapsed_time(e1), "iters": info.iters, "rel_residual": info.rel_residual,
                             "beta": beta, "sigma_v": 5.0, "bias": 1.0, "deflate": deflate_of(defl, n)}
    del s_m
    # the 3D mask from a sky map: 1024 x 512 pixels (a 30-degree cap of completeness 0.9 around
    # the survey axis) and the radial law tabulated every 0.25 Mpc/h to 500 Mpc/h: 1e9 ray samples
    na, nd, nr, dr = 1024, 512, 2000, 0.25
    al = (np.arange(na) + 0.5) * 2 * np.pi / na
    de = -np.pi / 2 + (np.arange(nd) + 0.5) * np.pi / nd
    ax = np.asarray(pr.sel.axis, dtype=np.float64)
    dot = (np.cos(de)[:, None] * np.cos(al)[None, :] * ax[0] + np.cos(de)[:, None] * np.sin(al)[None, :] * ax[1]
           + np.sin(de)[:, None] * ax[2])
    sky = torch.from_numpy(np.where(dot >= np.cos(pr.sel.half_angle), 0.9, 0.0)).to(s_rec.device)
    rr = (np.arange(nr) + 0.5) * dr
    p, kind = pr.sel.radial_params, pr.sel.radial_kind
    if kind == 0:
        wr = np.ones_like(rr)
    elif kind == 1:
        wr = np.exp(-(rr / p[0]) ** 2)
    else:
        wr = np.clip((rr / p[0]) ** p[1] * np.exp(p[1] * (1.0 - rr / p[0])), 0.0, 1.0)
    ms, _ = timed(lambda: ctx.project_mask(sky, n, box, 0.0, 2 * np.pi / na, -np.pi / 2, np.pi / nd,
                                           pr.sel.observer, dr, wr), reps=2)
    out["mask_projection"] = {"ms": ms, "samples": na * nd * nr, "gsamples_per_s": na * nd * nr / (ms * 1e6)}
    ctx.smooth(s_rec, box, 10.0, out=sm)
    shells = [[0.0, 200.0], [200.0, 400.0], [400.0, float("inf")], [0.0, 600.0]]
    obs = pr.sel.observer
    ms, (hist, mom) = timed(lambda: ctx.density_stats(sm, w, box, obs, shells, -1.0, 0.03, 200))
    out["density"] = {"ms": ms, "gbs": 16.0 * n ** 3 / (ms * 1e6),
                      "r10_skewness_obs_unobs": [[round(float(mom[s, g, 5]), 4) for g in (0, 1)] for s in range(4)],
                      "r10_kurtosis_obs_unobs": [[round(float(mom[s, g, 6]), 4) for g in (0, 1)] for s in range(4)],
                      "r10_pearson_obs_unobs": [[round(float(mom[s, g, 7]), 4) for g in (0, 1)] for s in range(4)]}
    return out


def bench_batch(ctx, dev, defl=0):
    import torch
    import paper_0906_3978_gb300 as wf
    mocks = batch_mocks()
    pos_d = [torch.from_numpy(m[3]).to(dev) for m in mocks]

    def prepare():
        probs = []
        for (n, box, sel, pos, k, p), pd in zip(mocks, pos_d):
            nobs = ctx.grid_assign(pd, n, box, wf.TSC, 2)
            w, d, b, nbar = ctx.build_noise(sel, nobs, pos.shape[0], box, want_d=False)
            probs.append(dict(w=w, nbar=nbar, b=b, box=box, pk_k=k, pk_p=p, tol=1e-6, max_iter=20000,
                              prec=wf.MIXED, deflate=defl))
        return probs

    probs = prepare()
    ctx.solve_batch(probs)            # warm-up (workspaces, tables)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    probs = prepare()
    torch.cuda.synchronize()
    t_prep = time.perf_counter() - t0
    st, outs, infos = ctx.solve_batch(probs)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t_batch_solve = t_batch - t_prep

    # the same work (gridding + window/noise + solve, same tolerance), one system after another:
    # plain FP64, and mixed precision without batching
    def sequential(prec):
        for (n, box, sel, pos, k, p), pd in zip(mocks[:2], pos_d[:2]):   # warm each path once
            nobs = ctx.grid_assign(pd, n, box, wf.TSC, 2)
            w, d, b, nbar = ctx.build_noise(sel, nobs, pos.shape[0], box, want_d=False)
            ctx.solve(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=prec,
                      deflate=defl if prec == wf.MIXED else 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (n, box, sel, pos, k, p), pd in zip(mocks, pos_d):
            nobs = ctx.grid_assign(pd, n, box, wf.TSC, 2)
            w, d, b, nbar = ctx.build_noise(sel, nobs, pos.shape[0], box, want_d=False)
            ctx.solve(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=prec,
                      deflate=defl if prec == wf.MIXED else 0)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_seq64 = sequential(wf.FP64)
    t_seqmix = sequential(wf.MIXED)
    sizes = {}
    for m in mocks:
        sizes[m[0]] = sizes.get(m[0], 0) + 1
    return {"workload": "96 mocks, N in {64,96,128,192} (counts %s), L = 1.953 N Mpc/h, 1e4-1e5 galaxies; "
                        "gridding + window/noise + one wf_solve_batch (mixed, FP32 inner / FP64 refinement) "
                        "to 1e-6; coarse radius by size (%s)" % (sizes, defl_note(defl)),
            "value": len(mocks) / t_batch, "unit": "solves/s", "status": st,
            "solve_only": {"value": len(mocks) / t_batch_solve, "unit": "solves/s"},
            "max_rel_residual": max(i.rel_residual for i in infos),
            "fp64_sequential": {"value": len(mocks) / t_seq64, "unit": "solves/s",
                                "note": "the same work (gridding + window/noise + plain FP64 wf_solve), one "
                                        "system at a time, same tolerance"},
            "mixed_sequential": {"value": len(mocks) / t_seqmix, "unit": "solves/s",
                                 "note": "the same work with mixed-precision wf_solve, one system at a time"}}


# ------------------------------------------------------------------------------------------
# Signal-dependent-noise Wiener filter with the Jackknife-like subsamples, at the mock setting of
# the paper's tests: 128^3 over 500 Mpc/h, ~2.2e5 galaxies, alpha = 1e-3, 200 reconstructions
# ------------------------------------------------------------------------------------------
def bench_jackknife(ctx, dev, defl=0, n=128, box=500.0, n_gal=218020, n_sub=200, alpha=1e-3, seed=4001):
    import numpy as np
    import torch
    import paper_0906_3978_gb300 as wf
    import synth
    k, p = synth.lcdm_table()
    sel = synth.selection_sdss_like(box, seed)
    pos = synth._cached_catalogue("jk_n%d_g%d_s%d" % (n, n_gal, seed),
                                  lambda: synth.lognormal_catalogue(n, box, k, p, sel, n_gal, seed))
    pd = torch.from_numpy(pos).to(dev)
    nobs = ctx.grid_assign(pd, n, box, wf.TSC, 2)
    w, d, b, nbar = ctx.build_noise(sel, nobs, pos.shape[0], box, want_d=False)
    wg = ctx.selection_eval(sel, pd)
    plain = {}
    for name, prec in (("fp64", wf.FP64), ("mixed", wf.MIXED)):
        dk = defl if prec == wf.MIXED else 0
        ctx.solve(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=prec, deflate=dk)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s, info = ctx.solve(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=prec, deflate=dk)
        torch.cuda.synchronize()
        plain[name] = {"solves_per_s": 1.0 / (time.perf_counter() - t0), "iters": info.iters}
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    u = torch.rand((n_sub, pos.shape[0]), dtype=torch.float64, device=dev, generator=gen)
    ctx.jackknife_solve(pd, wg, u[:8].contiguous(), alpha, nobs, w, nbar, n, box, k, p, tol=1e-6, max_iter=20000,
                        prec=wf.MIXED, check=False, deflate=defl)  # warm-up: workspaces of a batch of 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sm, infos = ctx.jackknife_solve(pd, wg, u, alpha, nobs, w, nbar, n, box, k, p, tol=1e-6, max_iter=20000,
                                    prec=wf.MIXED, check=False, deflate=defl)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    its = np.array([i.iters for i in infos])
    return {"workload": "%d^3 over %.0f Mpc/h, %d galaxies (SDSS-like cone and holes), alpha = %g, %d Jackknife-like "
                        "subsamples (one uniform per galaxy and subsample), signal-dependent-noise Wiener filter each "
                        "(lambda = N''), mixed precision to 1e-6 with coarse radius %s, mean of the reconstructions; "
                        "the plain filter's mixed solve with coarse radius %s" % (
                            n, box, pos.shape[0], alpha, n_sub, deflate_of(defl, n), deflate_of(defl, n)),
            "value": n_sub / t, "unit": "solves/s", "s": t, "ok": int(sum(1 for i in infos if i.status == 0)),
            "iters": {"min": int(its.min()), "median": int(np.median(its)), "max": int(its.max())},
            "plain_filter": plain,
            "note": "iterations against the plain filter's on the same catalogue measure the conditioning the "
                    "subsamples' sparse N'' gives the signal-dependent noise term"}


# ------------------------------------------------------------------------------------------
# Served form: Poisson stream of requests through wf_submit / wf_poll
# ------------------------------------------------------------------------------------------
SERVE_SIZES = [64, 72, 96, 108, 128, 144, 192, 216, 256, 288, 384]


def bench_serving(ctx, dev, defl=0, n_req=600, rate=20.0, seed=7):
    import numpy as np
    import torch
    import paper_0906_3978_gb300 as wf
    import synth
    rng = np.random.default_rng(seed)
    k, p = synth.lcdm_table()
    pool = {}
    for i, n in enumerate(SERVE_SIZES):     # one problem per size, shared by that size's requests
        box = 1.953 * n
        sel = synth.selection_sdss_like(box, seed + i, half_angle_deg=float(rng.uniform(20, 45)),
                                        r_peak=float(rng.uniform(100, 200)) * box / 500.0)
        ng = 0.009 * n ** 3 * float(rng.uniform(0.5, 1.5))
        pos = synth._cached_catalogue("serve_n%d_s%d" % (n, seed + i),
                                      lambda: synth.lognormal_catalogue(n, box, k, p, sel, ng, seed + i))
        nobs = ctx.grid_assign(torch.from_numpy(pos).to(dev), n, box, wf.TSC, 2)
        w, d, b, nbar = ctx.build_noise(sel, nobs, pos.shape[0], box, want_d=False)
        pool[n] = (w.cpu().numpy().copy(), b.cpu().numpy().copy(), nbar, box)
    sizes = rng.choice(SERVE_SIZES, size=n_req)
    gaps = rng.exponential(1.0 / rate, size=n_req)
    # FP64 comparison: service time of one plain FP64 solve per size
    t64 = {}
    for n in SERVE_SIZES:
        w, b, nbar, box = pool[n]
        wd, bd = torch.from_numpy(w).to(dev), torch.from_numpy(b).to(dev)
        ctx.solve(wd, nbar, bd, box, k, p, tol=1e-6, max_iter=20000, prec=wf.FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve(wd, nbar, bd, box, k, p, tol=1e-6, max_iter=20000, prec=wf.FP64)
        torch.cuda.synchronize()
        t64[n] = time.perf_counter() - t0
    # warm the serving path once per size
    for n in SERVE_SIZES:
        w, b, nbar, box = pool[n]
        ctx.poll(ctx.submit(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=wf.MIXED, deflate=defl), timeout_ms=-1)
    lat, stats = [], []
    t_start = time.perf_counter()
    submitted = []
    for i in range(n_req):
        target = t_start + float(np.sum(gaps[:i + 1]))
        now = time.perf_counter()
        if target > now:
            time.sleep(target - now)
        w, b, nbar, box = pool[int(sizes[i])]
        submitted.append(ctx.submit(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=wf.MIXED, deflate=defl))
    for rid in submitted:
        st, info = ctx.poll(rid, timeout_ms=-1)
        stats.append(st)
        lat.append(info.latency_s)
    t_total = time.perf_counter() - t_start
    lat = np.array(lat)
    mean64 = float(np.mean([t64[int(n)] for n in sizes]))
    # capacity: the first n_sat requests of the same size mix, all submitted at t = 0
    n_sat = n_req // 2
    t0 = time.perf_counter()
    ids = []
    for i in range(n_sat):
        w, b, nbar, box = pool[int(sizes[i])]
        ids.append(ctx.submit(w, nbar, b, box, k, p, tol=1e-6, max_iter=20000, prec=wf.MIXED, deflate=defl))
    sat_lat, sat_ok = [], 0
    for rid in ids:
        st, info = ctx.poll(rid, timeout_ms=-1)
        sat_ok += st == 0
        sat_lat.append(info.latency_s)
    t_sat = time.perf_counter() - t0
    return {"workload": "%d requests, Poisson arrivals at %.0f/s, N uniform over %s, L = 1.953 N Mpc/h, "
                        "0.009 N^3 x U(0.5,1.5) galaxies, random cone 20-45 deg and radial peak; mixed "
                        "precision to 1e-6 through wf_submit/wf_poll; coarse radius %s"
                        % (n_req, rate, SERVE_SIZES, defl_note(defl)),
            "value": n_req / t_total, "unit": "solves/s", "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "ok": int(sum(1 for s in stats if s == 0)),
            "capacity": {"value": n_sat / t_sat, "unit": "solves/s", "requests": n_sat, "ok": int(sat_ok),
                         "p50_s": float(np.percentile(sat_lat, 50)), "p99_s": float(np.percentile(sat_lat, 99)),
                         "note": "all requests submitted at once: the served throughput at saturation"},
            "fp64_sequential": {"value": 1.0 / mean64, "unit": "solves/s",
                                "note": "1 / mean service time of one plain FP64 wf_solve over the same size mix"}}


def deflate_of(defl, n):
    """The coarse radius a mixed solve of size n runs with for the option value defl (-1: the
    library's rule, wf_deflate_radius)."""
    if defl != -1:
        return defl
    import paper_0906_3978_gb300 as wf
    return wf.deflate_radius(n)


def defl_note(defl):
    return ("by grid size (0 below 64, 3 at 64, 4 to 128, 6 to 192, 8 to 256, 10 to 384, 12 above)" if defl == -1
            else str(defl))


def read_profile(ctx):
    return ctx.profile_read()


def cpu_full():
    """Whole oracle reconstructions of the 64^3 (tol 1e-8) and 256^3 (tol 1e-6) workloads on all host
    threads and on one.  The one-thread 256^3 figure is a whole solve only if it finishes within an
    hour's budget; otherwise it is scaled from the all-thread solve by the one-thread / all-thread
    time of one 256^3 matvec, and says so."""
    import numpy as np
    import oracle
    import synth
    oracle.build()
    nt = oracle.threads()
    out = {"kind": "oracle", "cpu": cpu_model(), "threads": nt}
    for name in ("c1", "c2"):
        t_all, it, rel = oracle_full_solve(name, nt)
        rec = {"workload": WORKLOADS[name], "cg_iters": it, "rel_residual": rel, "s": t_all,
               "solves_per_s": 1.0 / t_all}
        if name == "c1":
            t_one, _, _ = oracle_full_solve(name, 1)
            rec.update({"s_1_thread": t_one, "solves_per_s_1_thread": 1.0 / t_one})
        else:
            pr = synth.problem(name)
            tab = oracle.sinv_table(pr.n, pr.box, pr.pk_k, pr.pk_p)
            w = np.ones((pr.n,) * 3)
            t0 = time.perf_counter()
            oracle.matvec(tab, 0.05, w, w)
            mv_all = time.perf_counter() - t0
            oracle.set_threads(1)
            try:
                t0 = time.perf_counter()
                oracle.matvec(tab, 0.05, w, w)
                mv_one = time.perf_counter() - t0
            finally:
                oracle.set_threads(nt)
            rec.update({"s_1_thread": t_all * mv_one / mv_all, "extrapolated_1_thread": True,
                        "note_1_thread": "the all-thread solve x (one-thread / all-thread time of one matvec: "
                                         "%.2f / %.2f s)" % (mv_one, mv_all)})
            rec["solves_per_s_1_thread"] = 1.0 / rec["s_1_thread"]
        out[name] = rec
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wf", choices=["wf", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-forms", dest="no_forms", action="store_true",
                    help="leave out the batched and served forms (reported after the timed 512^3 steps)")
    ap.add_argument("--deflate", type=int, default=-1,
                    help="coarse radius of the mixed solves (-1: by grid size, 12 at 512^3; 0: none)")
    ap.add_argument("--cpu-full", dest="cpu_full", action="store_true",
                    help="only time whole oracle reconstructions of the 64^3 and 256^3 workloads on the host "
                         "(all threads and one thread) and print them as one JSON line")
    args = ap.parse_args()
    if args.cpu_full:
        return cpu_full()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
