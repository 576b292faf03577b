#!/usr/bin/env python
"""Throughput of the Fast Template Periodogram on one GB300 (or N, one per rank).

Workload: the single long lightcurve - N_obs = 1e4 times over a 3000 d
baseline with nightly gaps, an H = 6 template, N_f = 2.5e5 frequencies
f_k = k / (5 * 3000 d) - synthetic and seeded (synth.long_curve).  A step is
one ftp_periodogram call over the whole grid: NFFT sums, polynomial assembly,
roots, candidates.  `value` is mixed-precision (frequency x template)
evaluations per second with the inputs resident in HBM, L2 flushed between
steps; the FP64 path is timed beside it and their largest |dP| over every
frequency is reported.  `e2e` is the same metric through the C ABI with
pinned host buffers (copies inside the timed region).  `cpu_baseline` times
the FP64 CPU oracle on a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("FTP freq·template evals/s on 1 GB300, mixed vs FP64 at |ΔP|≤1e-4; "
          "%roofline")
UNIT = "evals/s"
WORKLOAD = ("single long lightcurve: N_obs=1e4 over 3000 d with nightly gaps (8 h windows, "
            "30% nights dropped), H=6 template, N_f=2.5e5, df=1/(5*3000 d)")
# HBM copy rate when no measured value is at hand (the profiling recipe's
# fallback for these GPUs); the ALU peaks are measured by every run.
HBM_FALLBACK_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20
# batch tuning cache (ftp_batch_autotune), outside the repository
TUNING_CACHE = os.environ.get("FTP_TUNING_CACHE",
                              os.path.join(os.path.expanduser("~"), ".cache", "ftp_gb300",
                                           "batch_tuning.json"))


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=128,
                    help="frequencies of the workload timed on the CPU oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 path (0 skips it)")
    ap.add_argument("--n-freq", type=int, default=None,
                    help="frequencies of the grid of the long and bank workloads (default "
                         "2.5e5 and 1e6; smaller only for profiling captures)")
    ap.add_argument("--workload", choices=["long", "survey", "bank", "screen", "small", "hsweep"],
                    default="long",
                    help="long: one long lightcurve (the headline line); survey: 4096 "
                         "curves batched; bank: 32 templates over one N=1e5 lightcurve; "
                         "screen: surrogate-screened survey vs exhaustive, with training; "
                         "small: the N=200, H=3, 5000-frequency curve, GPU vs the oracle's "
                         "CPU seconds on the whole grid; hsweep: time per evaluation vs H "
                         "on the long curve")
    ap.add_argument("--ncurves", type=int, default=4096, help="curves of the survey workload")
    ap.add_argument("--train-curves", type=int, default=50_000,
                    help="training curves of the screen workload")
    ap.add_argument("--heldout-curves", type=int, default=2048,
                    help="held-out curves of the screen workload")
    ap.add_argument("--train-steps", type=int, default=4000,
                    help="Adam steps of the screen workload's training")
    ap.add_argument("--train-cap", type=int, default=250_000_000,
                    help="training rows held on the device (screen workload)")
    return ap.parse_args()


# ------------------------------------------------------------------ oracle on CPU
def _oracle_worker(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    import numpy as np

    import oracle
    t, y, dy, freqs, c, s = args
    r = oracle.periodogram(t, y, dy, freqs, c, s)
    return r["power"]


def oracle_timing(lc, tpl, freqs, cores):
    """Time the FP64 oracle over `freqs` with a spawn pool of `cores` single-
    threaded workers; returns (seconds, powers)."""
    import numpy as np
    chunks = [c for c in np.array_split(freqs, max(1, cores * 2)) if c.size]
    jobs = [(lc.t, lc.y, lc.dy, ch, tpl.c, tpl.s) for ch in chunks]
    dt, parts = oracle_jobs(jobs, cores)
    return dt, np.concatenate(parts)


def oracle_jobs(jobs, cores):
    """Time oracle jobs (t, y, dy, freqs, c, s) on a spawn pool of `cores`
    single-threaded workers; returns (seconds, [powers per job])."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        with ctx.Pool(cores) as pool:
            j0 = jobs[0]
            pool.map(_oracle_worker, [(j0[0], j0[1], j0[2], j0[3][:1], j0[4], j0[5])] * cores)
            t0 = time.perf_counter()
            parts = pool.map(_oracle_worker, jobs)
            dt = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return dt, parts


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float, device) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, value: float, device) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"ftp_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def solver_report(stats, mean_iterations=None):
    """Root-solver counts of the last call: items that hit the Aberth cap in
    the main pass (before) and after their re-solve, and
    the frequencies re-solved from direct FP64 sums."""
    it = stats["mean_iterations"] if mean_iterations is None else mean_iterations
    return {"mean_iterations": round(it, 3),
            "nonconverged_before_resolve": stats["nonconverged"],
            "nonconverged_after_resolve": stats["still_nonconverged"],
            "resolved_frequencies": stats["resolved"],
            "resolved_for_nonconvergence": stats["resolved_nonconverged"]}


def ncu_traffic_per_item():
    """DRAM bytes per (frequency, template) item of the roots kernel, from the
    committed ncu summary (None if absent)."""
    p = os.path.join(ROOT, "profiles", "roots_kernel_long_curve.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.strip().startswith("dram_bytes_per_item:"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


# ------------------------------------------------------------------ peaks
def hbm_peak():
    """(GB/s, source) of the HBM copy rate measured on this machine's GPUs, else
    the recipe's fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def measure_alu_peaks(ftp, local):
    """Peak FP32, packed-FP32 and FP64 FMA rates of this GPU (TFLOP/s, best of
    three launches of ftp_alu_peak), with the SM clock sampled meanwhile."""
    iters = {0: 40_000, 1: 20_000, 2: 3_000}
    best = {}
    with ClockSampler(local) as clk:
        for kind, n in iters.items():
            rates = []
            for _ in range(3):
                flops, ms = ftp.ftp_alu_peak(local, kind, n)
                rates.append(flops / (ms / 1e3) / 1e12)
            best[kind] = max(rates)
    c = clk.summary() or {}
    out = {"fp32_tflops": round(best[0], 2), "fp32x2_tflops": round(best[1], 2),
           "fp64_tflops": round(best[2], 3), "sm_mhz": c.get("sm_mhz"),
           "how": "ftp_alu_peak: independent FMA chains on every SM (32 warps each), best of 3 "
                  "launches, CUDA events"}
    # the root kernels issue both scalar and packed FP32 FMAs: the larger rate bounds them
    out["fp32_peak_tflops"] = max(out["fp32_tflops"], out["fp32x2_tflops"])
    return out


def alu_roofline(achieved, peaks, kernel, traffic=None, traffic_note=None):
    peak = peaks["fp32_peak_tflops"]
    r = {"bound": "alu", "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
         "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kernel,
         "peak_source": f"measured in this run (FP32 FMA chains, ftp_alu_peak) at "
                        f"{peaks.get('sm_mhz')} MHz SM clock"}
    if traffic_note:
        r["traffic_note"] = traffic_note
    return r


# ------------------------------------------------------------------ our arm
def run_ours(args, world, rank, local, pg):
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp, shard

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # one lightcurve per rank: rank r analyses its own seeded curve of the
    # workload's shape (curves are independent: no data exchange)
    lc, tpl, grid = synth.long_curve(nf=args.n_freq or 250_000, seed=1002 + 1000 * rank)
    nf, D = grid.nf, 6 * tpl.H - 2
    stream = torch.cuda.Stream(device=dev)
    tpls = [(tpl.c, tpl.s)]
    dt_, dy_, ds_ = (torch.from_numpy(a).to(dev) for a in (lc.t, lc.y, lc.dy))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peaks = measure_alu_peaks(ftp, local)
    hbm, hbm_src = hbm_peak()

    def outputs():
        return ([torch.empty(nf, dtype=torch.float64, device=dev) for _ in range(4)],
                torch.empty(nf, dtype=torch.uint8, device=dev))

    def timed(plan, steps, warmup, outs, fl):
        """Device time of each of `steps` calls (stage timing off)."""
        for _ in range(warmup):
            ftp.ftp_periodogram(plan, dt_, dy_, ds_, lc.t.size, tpls, *outs, fl)
        return _timed_calls(stream, flush, steps, lambda: ftp.ftp_periodogram(
            plan, dt_, dy_, ds_, lc.t.size, tpls, *outs, fl))

    def staged(plan, calls, outs, fl):
        """Stage times, first-kernel time and iterations of `calls` timed calls."""
        ftp.ftp_set_timing(plan, True)
        st, first, iters = [], [], []
        with torch.cuda.stream(stream):
            for _ in range(calls):
                flush.zero_()
                ftp.ftp_periodogram(plan, dt_, dy_, ds_, lc.t.size, tpls, *outs, fl)
                st.append(ftp.ftp_stage_times(plan))
                first.append(ftp.ftp_roots_first_phase_ms(plan))
                iters.append(ftp.ftp_solver_stats(plan)["mean_iterations"])
        ftp.ftp_set_timing(plan, False)
        return np.array(st), first, iters

    sh = stream.cuda_stream
    mixed = ftp.ftp_plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, "mixed", local, sh)
    fp64 = ftp.ftp_plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, "fp64", local, sh)
    out_m, fl_m = outputs()
    out_d, fl_d = outputs()

    # ---- mixed, device-resident inputs: the headline (stage timing off)
    barrier(pg)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        step_ms = timed(mixed, args.steps, args.warmup, out_m, fl_m)
    torch.cuda.synchronize(dev)
    barrier(pg)
    clocks = clk.summary()
    launches_per_call = ftp.ftp_plan_info(mixed)["last_launches"]
    stats_m = ftp.ftp_solver_stats(mixed)
    total_ms = sum(step_ms)
    total_ms_max = max_over_ranks(pg, total_ms, dev)
    evals_all = sum_over_ranks(pg, float(args.steps * nf), dev)
    value = evals_all / (total_ms_max / 1e3)

    # ---- the stages, in separate calls with stage timing on
    st, first_ms, iters = staged(mixed, max(3, min(args.steps, 10)), out_m, fl_m)
    st_med = np.median(st, axis=0)
    first = statistics.median(first_ms)
    ibar = statistics.mean(iters)

    # ---- FP64 path beside it, and the mixed-vs-FP64 error on every frequency
    fp64_path = None
    if args.fp64_steps > 0:
        d_ms = timed(fp64, args.fp64_steps, 1, out_d, fl_d)
        fp64_path = {"value": round(nf * len(d_ms) / (sum(d_ms) / 1e3), 1), "unit": UNIT,
                     "steps": len(d_ms), "ms_per_step": round(statistics.mean(d_ms), 3),
                     "max_abs_dP_mixed_vs_fp64":
                         float(torch.max(torch.abs(out_m[0] - out_d[0])).item())}

    # ---- end to end through the C ABI with pinned host buffers
    th = [torch.from_numpy(a).pin_memory() for a in (lc.t, lc.y, lc.dy)]
    oh = [torch.empty(nf, dtype=torch.float64).pin_memory() for _ in range(4)]
    fh = torch.empty(nf, dtype=torch.uint8).pin_memory()
    ftp.ftp_periodogram(mixed, *th, lc.t.size, tpls, *oh, fh)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ftp.ftp_periodogram(mixed, *th, lc.t.size, tpls, *oh, fh)
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0, dev)
    e2e_value = evals_all / e2e_s
    h2d = 3 * lc.t.size * 8 + 16 * 16 + 4
    d2h = 4 * nf * 8 + nf + 8 * 4 * 2

    # ---- roofline of the dominant kernel: the first root-stage kernel
    #      (assembly, Aberth iterations, candidates), timed with events
    fp32_flops = nf * 26.0 * D * D * ibar          # Aberth: 26 D^2 flops per iteration
    achieved = fp32_flops / (first / 1e3) / 1e12
    tpi = ncu_traffic_per_item()
    roofline = alu_roofline(
        achieved, peaks, "roots_kernel phase 1 (assembly + Aberth + candidates; FP32 Aberth "
        "flops 26*D^2*iterations)", round(tpi * nf) if tpi else None,
        "DRAM bytes per item from an ncu capture of the same kernel on the first 2e4 "
        "frequencies of this workload, scaled to the launch's 2.5e5 items" if tpi else None)

    # ---- whole step: T* = sum over stages of the time at their bound
    info = ftp.ftp_plan_info(mixed)
    n_grid, H = info["grid_len"], tpl.H
    b_a = 8 * n_grid + 16 * n_grid + 16 * 2 * H * (grid.k0 + nf) + 24 * H * nf
    b_p2 = (24 * H + 24 + 33) * nf
    t_a = b_a / (hbm * 1e9) * 1e3
    t_1 = fp32_flops / (peaks["fp32_peak_tflops"] * 1e12) * 1e3
    t_2 = b_p2 / (hbm * 1e9) * 1e3
    m_a = float(np.sum(st_med[:4]))
    m_1, m_2 = first, float(st_med[4]) - first
    t_step = statistics.median(step_ms)
    whole = {
        "t_star_ms": round(t_a + t_1 + t_2, 4), "t_ms": round(t_step, 4),
        "frac": round((t_a + t_1 + t_2) / t_step, 4),
        "stages": {"step_a_sums": {"t_star_ms": round(t_a, 4), "t_ms": round(m_a, 4),
                                   "bound": "hbm"},
                   "roots_phase1": {"t_star_ms": round(t_1, 4), "t_ms": round(m_1, 4),
                                    "bound": "alu"},
                   "roots_phase2": {"t_star_ms": round(t_2, 4), "t_ms": round(m_2, 4),
                                    "bound": "hbm"}},
        "model": "step (a): spread writes 8 B per grid cell, FFT one read + one write "
                 "(16 B per cell), gather reads 16 B per needed grid index and writes 24H B "
                 "per frequency; phase 1: 26 D^2 iterations FP32 flops per item at the "
                 "measured FP32 peak; phase 2: (24H + 57) B per item at the HBM peak "
                 f"({hbm:.0f} GB/s, {hbm_src}); stage times from separate calls with stage "
                 "timing on, T from the headline steps (median)"}

    # ---- host merge of the ranks' results: each curve's best peak
    k_best = int(torch.argmax(out_m[0]).item())
    best = {"rank": rank, "f_best": float(grid.freqs()[k_best]),
            "P_best": float(out_m[0][k_best].item())}
    merged = shard.gather_to_root(pg, best, rank, world)
    torch.cuda.synchronize(dev)

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(statistics.mean(step_ms), 4),
        "ms_per_step_median": round(t_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_obs": int(lc.t.size), "H": tpl.H, "n_freq": nf,
                   "templates": 1, "l2": "flushed between steps (512 MiB write)",
                   "stage_timing": "off in the timed steps; stages from separate calls",
                   "parallelism": (f"{world} ranks, one distinct seeded lightcurve each "
                                   "(independent problems, no data exchange)")
                   if world > 1 else "single GPU"},
        "fp64_path": fp64_path,
        "stage_ms": {"moments_binning": round(float(st_med[0]), 4),
                     "spread": round(float(st_med[1]), 4), "fft": round(float(st_med[2]), 4),
                     "gather": round(float(st_med[3]), 4),
                     "roots": round(float(st_med[4]), 4), "roots_phase1": round(first, 4),
                     "resolve": round(float(st_med[5]), 4)},
        "solver": solver_report(stats_m, ibar),
        "roofline": roofline,
        "whole_step": whole,
        "alu_peaks": peaks,
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "gpu_launches": args.steps * launches_per_call,
    }
    if world > 1 and rank == 0:
        result["ranks"] = merged

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        sel = np.linspace(0, nf - 1, args.cpu_sample).astype(np.int64)
        sec, pw = oracle_timing(lc, tpl, grid.freqs()[sel], cores)
        gp = out_m[0].cpu().numpy()[sel]
        result["cpu_baseline"] = {
            "value": round(sel.size / sec, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sel.size} evenly spaced frequencies of the workload "
                      f"({sec:.1f} s wall on {cores} single-threaded processes)",
            "max_abs_dP_mixed_vs_oracle": float(np.max(np.abs(gp - pw)))}
    ftp.ftp_destroy(mixed)
    ftp.ftp_destroy(fp64)
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ extra workloads
BATCH_SURVEY = ("batched survey: {n} lightcurves, N_obs lognormal (median 1000, clipped 50-20000), "
          "baselines U(100,3000) d, bank of 16 templates H in (2,4,6), one per curve, "
          "df=1/(5T), f<=10/d")
BANK = ("template bank over one long lightcurve: N_obs=1e5 over 4000 d with nightly gaps, "
        "32 templates H=10, N_f=1e6, df=1/(5*4000 d)")


def subset_survey(sv, idx):
    """The curves `idx` of a synthetic survey, as a survey of their own."""
    import numpy as np

    import synth
    idx = np.asarray(idx, dtype=np.int64)
    n = np.diff(sv.obs_off)[idx]
    off = np.zeros(idx.size + 1, dtype=np.int64)
    off[1:] = np.cumsum(n)
    sl = [np.arange(sv.obs_off[c], sv.obs_off[c + 1]) for c in idx]
    cat = np.concatenate(sl) if sl else np.zeros(0, dtype=np.int64)
    return synth.Survey(off, sv.t[cat], sv.y[cat], sv.dy[cat], [sv.grids[c] for c in idx],
                        sv.bank, sv.tpl_of_curve[idx], sv.injected[idx], sv.period[idx])


def _timed_calls(stream, flush, steps, call):
    """CUDA-event times (ms) of `steps` calls on `stream`, L2 flushed before each."""
    import torch
    out = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
    return out


def _result(args, world, metric_value, step_ms, cfg, scaling="weak", **extra):
    r = {"metric": METRIC, "value": round(metric_value, 1), "unit": UNIT, "n_gpus": world,
         "steps": args.steps, "warmup": args.warmup,
         "ms_per_step": round(statistics.mean(step_ms), 4),
         "ms_per_step_median": round(statistics.median(step_ms), 4), "higher_is_better": True,
         "scaling": scaling, "vs_baseline": None, "dtype": "f32+f64 (mixed)",
         "data": "synthetic", "config": cfg}
    r.update(extra)
    return r


def run_survey(args, world, rank, local, pg):
    import numpy as np
    import torch

    os.makedirs(os.path.dirname(TUNING_CACHE), exist_ok=True)
    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp

    from paper_2101_12348_gb300 import shard

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    full = synth.survey(ncurves=args.ncurves, seed=1003)
    # curves shared out across ranks, balanced by the root stage's cost
    # (frequencies x D^2); a single rank takes them all
    cost = np.array([g.nf * (6 * full.bank[full.tpl_of_curve[c]].H - 2) ** 2
                     for c, g in enumerate(full.grids)], dtype=np.float64)
    parts = shard.partition_by_cost(cost, world)
    mine = parts[rank]
    sv = subset_survey(full, mine)
    peaks = measure_alu_peaks(ftp, local)
    bank = [(b.c, b.s) for b in sv.bank]
    grids = [(g.df, g.k0, g.nf) for g in sv.grids]
    nfs = np.array([g.nf for g in sv.grids], dtype=np.int64)
    Hc = np.array([sv.bank[i].H for i in sv.tpl_of_curve])
    out_off = np.zeros(sv.ncurves + 1, dtype=np.int64)
    out_off[1:] = np.cumsum(nfs)
    tot = int(out_off[-1])
    gj = max(sv.grids, key=lambda g: g.k0 + g.nf)
    plan_grid = (gj.df, gj.k0, int(nfs.max()))
    max_nobs = int(np.max(np.diff(sv.obs_off)))
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    dt_, dy_, ds_ = (torch.from_numpy(a).to(dev) for a in (sv.t, sv.y, sv.dy))
    outs = [torch.empty(tot, dtype=torch.float64, device=dev) for _ in range(4)]
    fl = torch.empty(tot, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    plan = ftp.ftp_plan(max_nobs, 6, plan_grid, len(bank), "mixed", local, sh)

    def call():
        ftp.ftp_batch(plan, sv.obs_off, dt_, dy_, ds_, grids, out_off[:-1], bank,
                      sv.tpl_of_curve, *outs, fl)

    t_first = time.perf_counter()
    call()  # first call: FFT plans, workspace
    first_s = time.perf_counter() - t_first
    # autotune (untimed): step (a) lanes and the roots grid, cached per batch shape
    t_tune = time.perf_counter()
    tuning = ftp.ftp_batch_autotune(plan, sv.obs_off, dt_, dy_, ds_, grids, out_off[:-1], bank,
                                    sv.tpl_of_curve, *outs, cache_path=TUNING_CACHE)
    tuning["seconds"] = round(time.perf_counter() - t_tune, 2)
    for _ in range(max(0, args.warmup - 1)):
        call()
    barrier(pg)
    with ClockSampler(local) as clk:
        step_ms = _timed_calls(stream, flush, args.steps, call)
    barrier(pg)
    clocks = clk.summary()
    info = ftp.ftp_batch_info(plan)
    launches = ftp.ftp_plan_info(plan)["last_launches"]
    total_ms = max_over_ranks(pg, sum(step_ms), dev)
    value = sum_over_ranks(pg, float(args.steps * tot), dev) / (total_ms / 1e3)
    # one eager call with stage timing: the split between sums and roots
    ftp.ftp_set_timing(plan, True)
    call()
    st = ftp.ftp_stage_times(plan)
    stats = ftp.ftp_solver_stats(plan)
    ftp.ftp_set_timing(plan, False)
    ibar = stats["mean_iterations"]
    flops = float(np.sum(nfs * 26.0 * (6 * Hc - 2) ** 2)) * ibar
    achieved = flops / (st[4] / 1e3) / 1e12
    roofline = alu_roofline(achieved, peaks, "roots stage, both kernels (FP32 Aberth flops "
                            "26*D^2*iterations, summed over curves with the batch's mean "
                            "iteration count)")
    # FP64 path on the first 64 curves, and the mixed-vs-FP64 error there
    nsub = min(64, sv.ncurves)
    sub_tot = int(out_off[nsub])
    p64 = ftp.ftp_plan(max_nobs, 6, plan_grid, len(bank), "fp64", local, sh)
    o64 = [torch.empty(sub_tot, dtype=torch.float64, device=dev) for _ in range(4)]
    sub_off = sv.obs_off[:nsub + 1].copy()

    def call64():
        ftp.ftp_batch(p64, sub_off, dt_, dy_, ds_, grids[:nsub], out_off[:nsub], bank,
                      sv.tpl_of_curve[:nsub], *o64, None)

    call64()
    d_ms = _timed_calls(stream, flush, max(1, args.fp64_steps), call64)
    fp64_path = {"value": round(sub_tot * len(d_ms) / (sum(d_ms) / 1e3), 1), "unit": UNIT,
                 "curves": nsub, "ms_per_step": round(statistics.mean(d_ms), 3),
                 "max_abs_dP_mixed_vs_fp64":
                     float(torch.max(torch.abs(outs[0][:sub_tot] - o64[0])).item())}
    ftp.ftp_destroy(p64)
    del o64
    # end to end: pinned host inputs and outputs, copies inside the timed region
    th = [torch.from_numpy(a).pin_memory() for a in (sv.t, sv.y, sv.dy)]
    oh = [torch.empty(tot, dtype=torch.float64).pin_memory() for _ in range(4)]
    fh = torch.empty(tot, dtype=torch.uint8).pin_memory()

    def call_host():
        ftp.ftp_batch(plan, sv.obs_off, *th, grids, out_off[:-1], bank, sv.tpl_of_curve, *oh, fh)

    call_host()
    e2e_steps = min(3, args.steps)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        call_host()
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0, dev)
    e2e = {"value": round(sum_over_ranks(pg, float(e2e_steps * tot), dev) / e2e_s, 1),
           "unit": UNIT, "h2d_bytes_per_step": int(3 * sv.t.size * 8),
           "d2h_bytes_per_step": int(tot * 33), "steps": e2e_steps}
    # host merge: each curve's best power, back in survey order on rank 0
    best_c = np.array([float(outs[0][out_off[c]:out_off[c + 1]].max().item())
                       for c in range(sv.ncurves)])
    got = shard.gather_to_root(pg, (mine, best_c), rank, world)
    cfg = {"workload": BATCH_SURVEY.format(n=full.ncurves), "curves": full.ncurves,
           "curves_this_rank": sv.ncurves,
           "n_obs_total": int(sv.t.size), "evals_per_step": tot, "templates_per_curve": 1,
           "l2": "flushed between steps (512 MiB write); sum tiles exceed L2",
           "graph": {0: "eager", 1: "captured", 2: "replayed"}[info["graph"]],
           "chunks": info["chunks"],
           "parallelism": (f"{world} ranks, curves balanced by N_f*D^2 (no data exchange; "
                           "host merge of results)") if world > 1 else "single GPU"}
    if rank == 0 and world > 1:
        merged = shard.merge_parts(full.ncurves, got)
        cfg["merged_curves"] = int(merged.size)
        cfg["rank_loads"] = [round(float(x) / float(cost.sum()), 4)
                             for x in shard.part_loads(cost, parts)]
    result = _result(args, world, value, step_ms, cfg,
                     scaling="strong" if world > 1 else "weak", alu_peaks=peaks,
                     fp64_path=fp64_path,
                     stage_ms={"sums": round(st[0], 3), "roots": round(st[4], 3),
                               "resolve": round(st[5], 3)},
                     first_call_s=round(first_s, 3), autotune=tuning,
                     solver=solver_report(stats, ibar),
                     roofline=roofline, e2e=e2e, clocks=clocks,
                     gpu_launches=args.steps * launches)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        rng = np.random.default_rng(11)
        jobs, picks = [], []
        for c in rng.choice(sv.ncurves, 2 * cores, replace=False):
            lc, g, tp = sv.curve(c), sv.grids[c], sv.bank[sv.tpl_of_curve[c]]
            k = np.sort(rng.choice(g.nf, 4, replace=False))
            jobs.append((lc.t, lc.y, lc.dy, g.freqs()[k], tp.c, tp.s))
            picks.append(out_off[c] + k)
        sec, parts = oracle_jobs(jobs, cores)
        gp = outs[0].cpu().numpy()
        err = max(float(np.max(np.abs(gp[pk] - pw))) for pk, pw in zip(picks, parts))
        n = sum(len(pk) for pk in picks)
        result["cpu_baseline"] = {
            "value": round(n / sec, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"4 random frequencies of each of {len(jobs)} random curves "
                      f"({sec:.1f} s wall on {cores} single-threaded processes)",
            "max_abs_dP_mixed_vs_oracle": err}
    ftp.ftp_destroy(plan)
    if rank == 0:
        print(json.dumps(result), flush=True)


def run_bank(args, world, rank, local, pg):
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp

    from paper_2101_12348_gb300 import shard

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lc, bank_all, grid = synth.bank_curve(nf=args.n_freq or 1_000_000)
    # templates shared out across ranks (r, r + world, ...): each rank runs
    # its templates on the whole grid; the sums are recomputed per rank
    mine = shard.partition_strided(len(bank_all), world)[rank]
    bank_t = [bank_all[i] for i in mine]
    peaks = measure_alu_peaks(ftp, local)
    bank = [(b.c, b.s) for b in bank_t]
    H, ntpl, nf = bank_t[0].H, len(bank), grid.nf
    D = 6 * H - 2
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    dt_, dy_, ds_ = (torch.from_numpy(a).to(dev) for a in (lc.t, lc.y, lc.dy))
    outs = [torch.empty(ntpl * nf, dtype=torch.float64, device=dev) for _ in range(4)]
    fl = torch.empty(ntpl * nf, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    plan = ftp.ftp_plan(lc.t.size, H, (grid.df, grid.k0, nf), ntpl, "mixed", local, sh)

    def call():
        ftp.ftp_periodogram(plan, dt_, dy_, ds_, lc.t.size, bank, *outs, fl)

    for _ in range(args.warmup):
        call()
    barrier(pg)
    with ClockSampler(local) as clk:
        step_ms = _timed_calls(stream, flush, args.steps, call)
    barrier(pg)
    clocks = clk.summary()
    stats = ftp.ftp_solver_stats(plan)
    # stage split in separate calls with stage timing on
    ftp.ftp_set_timing(plan, True)
    roots, sums, first = [], [], []
    for _ in range(max(2, min(args.steps, 5))):
        _timed_calls(stream, flush, 1, call)
        st = ftp.ftp_stage_times(plan)
        roots.append(st[4])
        first.append(ftp.ftp_roots_first_phase_ms(plan))
        sums.append(st[0] + st[1] + st[2] + st[3])
    ftp.ftp_set_timing(plan, False)
    launches = ftp.ftp_plan_info(plan)["last_launches"]
    total_ms = max_over_ranks(pg, sum(step_ms), dev)
    evals = ntpl * nf
    value = sum_over_ranks(pg, float(args.steps * evals), dev) / (total_ms / 1e3)
    ibar = stats["mean_iterations"]
    achieved = evals * 26.0 * D * D * ibar / (statistics.mean(first) / 1e3) / 1e12
    roofline = alu_roofline(achieved, peaks, "roots_kernel phase 1 (assembly + Aberth + "
                            "candidates; FP32 Aberth flops 26*D^2*iterations)")
    # FP64 path on the first 20000 frequencies (all 32 templates)
    nf64 = min(20_000, nf)
    p64 = ftp.ftp_plan(lc.t.size, H, (grid.df, grid.k0, nf64), ntpl, "fp64", local, sh)
    o64 = [torch.empty(ntpl * nf64, dtype=torch.float64, device=dev) for _ in range(4)]

    def call64():
        ftp.ftp_periodogram(p64, dt_, dy_, ds_, lc.t.size, bank, *o64, None)

    call64()
    d_ms = _timed_calls(stream, flush, max(1, args.fp64_steps), call64)
    pm = outs[0].view(ntpl, nf)[:, :nf64]
    fp64_path = {"value": round(ntpl * nf64 * len(d_ms) / (sum(d_ms) / 1e3), 1), "unit": UNIT,
                 "n_freq": nf64, "ms_per_step": round(statistics.mean(d_ms), 3),
                 "max_abs_dP_mixed_vs_fp64":
                     float(torch.max(torch.abs(pm - o64[0].view(ntpl, nf64))).item())}
    ftp.ftp_destroy(p64)
    th = [torch.from_numpy(a).pin_memory() for a in (lc.t, lc.y, lc.dy)]
    oh = [torch.empty(ntpl * nf, dtype=torch.float64).pin_memory() for _ in range(4)]
    fh = torch.empty(ntpl * nf, dtype=torch.uint8).pin_memory()
    ftp.ftp_periodogram(plan, *th, lc.t.size, bank, *oh, fh)
    e2e_steps = min(3, args.steps)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ftp.ftp_periodogram(plan, *th, lc.t.size, bank, *oh, fh)
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0, dev)
    e2e = {"value": round(sum_over_ranks(pg, float(e2e_steps * evals), dev) / e2e_s, 1),
           "unit": UNIT, "h2d_bytes_per_step": int(3 * lc.t.size * 8),
           "d2h_bytes_per_step": int(evals * 33), "steps": e2e_steps}
    best_t = outs[0].view(ntpl, nf).max(dim=1).values.cpu().numpy()
    got = shard.gather_to_root(pg, (mine, best_t), rank, world)
    cfg = {"workload": BANK, "n_obs": int(lc.t.size), "H": H, "templates": len(bank_all),
           "templates_this_rank": ntpl, "n_freq": nf,
           "l2": "flushed between steps (512 MiB write); sum tiles exceed L2",
           "parallelism": (f"{world} ranks, templates r, r+{world}, ... per rank (no data "
                           "exchange; host merge of results)") if world > 1 else "single GPU"}
    if rank == 0 and world > 1:
        cfg["merged_templates"] = int(shard.merge_parts(len(bank_all), got).size)
    result = _result(args, world, value, step_ms, cfg, fp64_path=fp64_path,
                     scaling="strong" if world > 1 else "weak", alu_peaks=peaks,
                     stage_ms={"sums": round(statistics.mean(sums), 3),
                               "roots": round(statistics.mean(roots), 3),
                               "roots_phase1": round(statistics.mean(first), 3)},
                     solver=solver_report(stats, ibar),
                     roofline=roofline, e2e=e2e, clocks=clocks,
                     gpu_launches=args.steps * launches)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        rng = np.random.default_rng(12)
        jobs, picks = [], []
        for i in rng.choice(ntpl, min(ntpl, cores), replace=False):
            k = np.sort(rng.choice(nf, 2, replace=False))
            jobs.append((lc.t, lc.y, lc.dy, grid.freqs()[k], bank_t[i].c, bank_t[i].s))
            picks.append(i * nf + k)
        sec, parts = oracle_jobs(jobs, cores)
        gp = outs[0].cpu().numpy()
        err = max(float(np.max(np.abs(gp[pk] - pw))) for pk, pw in zip(picks, parts))
        n = sum(len(pk) for pk in picks)
        result["cpu_baseline"] = {
            "value": round(n / sec, 2), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"2 random frequencies for each of {len(jobs)} templates "
                      f"({sec:.1f} s wall on {cores} single-threaded processes)",
            "max_abs_dP_mixed_vs_oracle": err}
    ftp.ftp_destroy(plan)
    if rank == 0:
        print(json.dumps(result), flush=True)


SMALL = ("single small lightcurve: N_obs=200 uniform in [0,30] d, H=3 template, "
         "f_k=k/150, k=1..5000; metric of this configuration: oracle CPU seconds")


def run_small(args, world, rank, local, pg):
    """The small curve: the whole grid on the GPU (mixed and FP64 paths) and
    on the CPU oracle (one process, and a spawn pool over every core), with
    |dP| against the oracle on every frequency."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lc, tpl, grid = synth.small_curve()
    nf = grid.nf
    tpls = [(tpl.c, tpl.s)]
    dt_, dy_, ds_ = (torch.from_numpy(a).to(dev) for a in (lc.t, lc.y, lc.dy))
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    res = {}
    for prec in ("mixed", "fp64"):
        plan = ftp.ftp_plan(lc.t.size, tpl.H, (grid.df, grid.k0, nf), 1, prec, local,
                            stream.cuda_stream)
        outs = [torch.empty(nf, dtype=torch.float64, device=dev) for _ in range(4)]

        def call():
            ftp.ftp_periodogram(plan, dt_, dy_, ds_, lc.t.size, tpls, *outs, None)

        for _ in range(max(3, args.warmup)):
            call()
        ms = _timed_calls(stream, flush, args.steps, call)
        res[prec] = (ms, outs[0].cpu().numpy())
        ftp.ftp_destroy(plan)
    freqs = grid.freqs()
    one_s, _ = oracle_timing(lc, tpl, freqs[: max(1, nf // 10)], 1)  # a tenth, scaled
    one_s *= nf / max(1, nf // 10)
    cores = cpu_cores()
    all_s, p_or = oracle_timing(lc, tpl, freqs, cores)
    ms_m, p_m = res["mixed"]
    ms_d, p_d = res["fp64"]
    value = nf / (statistics.mean(ms_m) / 1e3)
    result = _result(args, world, value, ms_m,
                     {"workload": SMALL, "n_obs": int(lc.t.size), "H": tpl.H, "n_freq": nf,
                      "l2": "flushed between steps (512 MiB write)", "parallelism": "single GPU"},
                     fp64_path={"value": round(nf / (statistics.mean(ms_d) / 1e3), 1),
                                "unit": UNIT, "ms_per_step": round(statistics.mean(ms_d), 4),
                                "max_abs_dP_vs_oracle": float(np.max(np.abs(p_d - p_or)))},
                     parity={"max_abs_dP_mixed_vs_oracle": float(np.max(np.abs(p_m - p_or))),
                             "max_abs_dP_fp64_vs_oracle": float(np.max(np.abs(p_d - p_or))),
                             "frequencies": nf},
                     cpu_baseline={"value": round(nf / all_s, 2), "unit": UNIT, "cores": cores,
                                   "kind": "oracle", "sample": "every frequency of the grid",
                                   "oracle_seconds_all_cores": round(all_s, 3),
                                   "oracle_seconds_one_core": round(one_s, 3)})
    print(json.dumps(result), flush=True)


def run_hsweep(args, world, rank, local, pg):
    """Time per (frequency, template) evaluation against the number of
    harmonics H = 1..16 on the long curve's observations (the paper's timing
    versus H): mixed path, 50 000 frequencies, stage split and iterations."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lc, _, grid = synth.long_curve(nf=50_000)
    nf = grid.nf
    dt_, dy_, ds_ = (torch.from_numpy(a).to(dev) for a in (lc.t, lc.y, lc.dy))
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    for H in range(1, 17):
        tpl = synth.make_template(H, 2000 + H)
        plan = ftp.ftp_plan(lc.t.size, H, (grid.df, grid.k0, nf), 1, "mixed", local,
                            stream.cuda_stream)
        outs = [torch.empty(nf, dtype=torch.float64, device=dev) for _ in range(4)]

        def call():
            ftp.ftp_periodogram(plan, dt_, dy_, ds_, lc.t.size, [(tpl.c, tpl.s)], *outs, None)

        for _ in range(max(2, args.warmup)):
            call()
        ms = _timed_calls(stream, flush, max(3, args.steps), call)
        ftp.ftp_set_timing(plan, True)
        call()
        st = ftp.ftp_stage_times(plan)
        it = ftp.ftp_solver_stats(plan)["mean_iterations"]
        ftp.ftp_set_timing(plan, False)
        ftp.ftp_destroy(plan)
        step = statistics.median(ms)
        rows.append({"H": H, "D": 6 * H - 2, "ms_per_step": round(step, 4),
                     "ns_per_eval": round(1e6 * step / nf, 2),
                     "sums_ms": round(sum(st[:4]), 4), "roots_ms": round(st[4], 4),
                     "mean_iterations": round(it, 2)})
    best = rows[5]
    result = _result(args, world, nf / (best["ms_per_step"] / 1e3), [best["ms_per_step"]],
                     {"workload": "H sweep: long-curve observations (N_obs=1e4), N_f=5e4, "
                                  "one seeded template per H = 1..16; value at H = 6",
                      "n_obs": int(lc.t.size), "n_freq": nf, "parallelism": "single GPU"},
                     sweep=rows)
    print(json.dumps(result), flush=True)


SCREEN = ("learned screening: {n} held-out lightcurves drawn as the batched survey with H=4 "
          "templates (bank of 16), surrogate 10->128->128->1 BF16 trained on exact FTP of "
          "{m} curves; exact solve on the top 1% of frequencies +-3 neighbours")


def run_screen(args, world, rank, local, pg):
    """Surrogate screening (2H+2 features -> BF16 MLP -> top 1% +- 3 -> exact
    solve) against the exhaustive batch on held-out curves.  Training data
    are exact GPU results on separate curves; training is untimed and
    reported.  A step is one screened batch over every held-out curve; value
    counts every frequency of those curves (the periodogram peak question is
    answered for all of them), exact_evals counts the ones solved exactly."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp, screen

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    H, nfeat, top, nbr = 4, 10, 0.01, 3
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    # plan large enough for every curve drawn as the survey (T <= 3000 d, N <= 20000)
    plan = ftp.ftp_plan(20_000, H, (1.0 / 15000.0, 1, 150_000), 16, "mixed", local, sh)
    # ---- training rows from exact results, 1024 curves at a time
    cap = args.train_cap  # rows (44 B each: features and label)
    Xt = torch.empty((cap, nfeat), dtype=torch.float32, device=dev)
    yt = torch.empty(cap, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    nrows, done, group = 0, 0, 0
    while done < args.train_curves:
        m = min(1024, args.train_curves - done)
        sv = synth.survey(ncurves=m, Hs=(H,), seed=50_000 + group)
        nrows = screen.training_rows(plan, sv.obs_off, sv.t, sv.y, sv.dy,
                                     [(g.df, g.k0, g.nf) for g in sv.grids],
                                     [(b.c, b.s) for b in sv.bank], sv.tpl_of_curve, H,
                                     top_frac=0.005, neighbours=3, rand_frac=0.005,
                                     seed=group + 1,
                                     X_out=Xt, y_out=yt, count=nrows)
        done += m
        group += 1
    rows = min(nrows, cap)
    torch.cuda.synchronize(dev)
    label_s = time.perf_counter() - t0
    net = screen.Surrogate(H, seed=3, device=local)
    losses = np.empty(args.train_steps, dtype=np.float32)
    t0 = time.perf_counter()
    net.train(Xt, yt, rows, steps=args.train_steps, batch=4096, lr=2e-3, seed=9, losses=losses)
    train_s = time.perf_counter() - t0
    del Xt, yt
    # ---- held-out curves: exhaustive vs screened
    sv = synth.survey(ncurves=args.heldout_curves, Hs=(H,), seed=90_001)
    bank = [(b.c, b.s) for b in sv.bank]
    grids = [(g.df, g.k0, g.nf) for g in sv.grids]
    off = screen.row_offsets(grids)
    tot = int(off[-1])
    dt_, dy_, ds_ = (torch.from_numpy(a).to(dev) for a in (sv.t, sv.y, sv.dy))
    ex = [torch.empty(tot, dtype=torch.float64, device=dev) for _ in range(4)]
    sc = [torch.empty(tot, dtype=torch.float64, device=dev) for _ in range(4)]
    fl = torch.empty(tot, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def call_ex():
        ftp.ftp_batch(plan, sv.obs_off, dt_, dy_, ds_, grids, off[:-1], bank, sv.tpl_of_curve,
                      *ex, None)

    def call_sc():
        ftp.ftp_batch_screened(plan, sv.obs_off, dt_, dy_, ds_, grids, off[:-1], bank,
                               sv.tpl_of_curve, net.h, top, nbr, *sc, fl)

    for _ in range(max(1, args.warmup)):
        call_sc()
    barrier(pg)
    with ClockSampler(local) as clk:
        step_ms = _timed_calls(stream, flush, args.steps, call_sc)
    barrier(pg)
    clocks = clk.summary()
    launches = ftp.ftp_plan_info(plan)["last_launches"]
    stats = ftp.ftp_solver_stats(plan)
    # one eager call with stage events: step (a) / screening / exact roots / re-solve
    ftp.ftp_set_timing(plan, True)
    call_sc()
    torch.cuda.synchronize(dev)
    st = ftp.ftp_stage_times(plan)
    ftp.ftp_set_timing(plan, False)
    stage = {"sums": round(st[0], 3), "screen": round(st[1], 3), "roots": round(st[4], 3),
             "resolve": round(st[5], 3)}
    call_ex()
    ex_ms = _timed_calls(stream, flush, max(1, min(3, args.steps)), call_ex)
    P_ex, P_sc = ex[0].cpu().numpy(), sc[0].cpu().numpy()
    evaluated = int(np.sum(~np.isnan(P_sc)))
    hits = []
    for c in range(sv.ncurves):
        a, b = P_sc[off[c]:off[c + 1]], P_ex[off[c]:off[c + 1]]
        hits.append(bool(np.nanmax(a) >= b.max() - 1e-4))
    recall = float(np.mean(hits))
    inj = sv.injected
    total_ms = max_over_ranks(pg, sum(step_ms), dev)
    value = sum_over_ranks(pg, float(args.steps * tot), dev) / (total_ms / 1e3)
    ex_value = tot * len(ex_ms) / (sum(ex_ms) / 1e3)
    cfg = {"workload": SCREEN.format(n=sv.ncurves, m=args.train_curves),
           "curves": sv.ncurves, "freqs_per_step": tot, "top_frac": top, "neighbours": nbr,
           "l2": "flushed between steps (512 MiB write)", "parallelism": "single GPU"}
    result = _result(args, world, value, step_ms, cfg,
                     screening={"recall": recall,
                                "recall_injected": float(np.mean(np.array(hits)[inj])),
                                "recall_noise": float(np.mean(np.array(hits)[~inj])),
                                "evaluated_frac": round(evaluated / tot, 4),
                                "exact_evals_per_s": round(evaluated * args.steps /
                                                           (total_ms / 1e3), 1),
                                "exhaustive_value": round(ex_value, 1),
                                "speedup_vs_exhaustive": round(value / ex_value, 3)},
                     training={"curves": args.train_curves, "rows": rows,
                               "rows_selected": nrows,
                               "selection": "exact top 0.5% +-3 and a random 0.5% of each "
                                            "curve's frequencies",
                               "label_s": round(label_s, 2), "train_s": round(train_s, 2),
                               "steps": args.train_steps, "batch": 4096,
                               "loss_first": float(losses[:20].mean()),
                               "loss_last": float(losses[-100:].mean())},
                     solver={"mean_iterations": round(stats["mean_iterations"], 3),
                             "items_last_call": stats["items"]},
                     stage_ms=stage, clocks=clocks, gpu_launches=args.steps * launches)
    net.close()
    ftp.ftp_destroy(plan)
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ reference arm
def run_reference(args, world, rank, local, pg):
    """The FP64 CPU oracle on the host cores, on the same workload and metric:
    each step is a bounded sample of frequencies of the workload."""
    if rank != 0:
        return
    import numpy as np

    import synth
    lc, tpl, grid = synth.long_curve()
    cores = cpu_cores()
    per_step = max(cores, 32)
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        oracle_timing(lc, tpl, grid.freqs()[rng.choice(grid.nf, cores, replace=False)], cores)
    secs, n = 0.0, 0
    for _ in range(args.steps):
        f = grid.freqs()[np.sort(rng.choice(grid.nf, per_step, replace=False))]
        s, _ = oracle_timing(lc, tpl, f, cores)
        secs += s
        n += f.size
    value = n / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * secs / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_obs": int(lc.t.size), "H": tpl.H,
                   "n_freq": grid.nf, "templates": 1},
        "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": f"{per_step} random frequencies of the workload per step"},
        "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse_args()
    world, rank, local, pg = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, local, pg)
        elif args.workload == "survey":
            run_survey(args, world, rank, local, pg)
        elif args.workload == "bank":
            run_bank(args, world, rank, local, pg)
        elif args.workload == "screen":
            run_screen(args, world, rank, local, pg)
        elif args.workload == "small":
            run_small(args, world, rank, local, pg)
        elif args.workload == "hsweep":
            run_hsweep(args, world, rank, local, pg)
        else:
            run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
