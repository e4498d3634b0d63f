#!/usr/bin/env python3
"""Benchmark: batched TaylorF2 lnL evaluations per second on one GB300 (or N, weak scaling).

Workload (one step): one gwl_loglike call over a batch of 8192 proposals for
a 3-detector, 8 s, 20-1024 Hz network (8033 bins per detector, coloured
Gaussian noise, 11-D aligned-spin BBH injection at SNR 15-30); half the
proposals are prior draws and half perturb the injection.  Inputs are
synthetic and seeded; the injection is produced by the device library's own
template (gwl_waveform), so the GPU leg runs no oracle code.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gwl|reference]

Prints one JSON line (rank 0).  ``value`` is the mixed-precision path's
device-timed throughput with inputs resident in HBM; L2 (129 MB) is flushed
by writing a 256 MB buffer between timed steps (the step inputs are < 1 MB).
``e2e`` is the same metric through gwl_loglike_host (host buffers, copies in
the timed region).  ``roofline`` refers to the dominant kernel (the windowed
bin loop), timed by the library's CUDA events on the launch stream.
``cpu_baseline`` times the FP64 oracle on the host cores on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_11873_gb300 import inputs as I  # noqa: E402

METRIC = "lnL evals/s (BBH 3-det 8s, 11-D)"
CONFIG = "c2"
BATCH = 8192
SEED = 2
# Algorithmic work per in-band (proposal, bin) pair with 3 detectors (flops,
# FMA = 2), counted from what the method must compute, not from the kernel's
# instructions: the phase, 9 basis terms (9 FMA = 18 flop) and per detector
# the delay term, nearest integer and subtraction (3 x 4 = 12 flop); the
# inner-product accumulation, 4 FMA per detector (24 flop), and its
# compensation (24 flop) -> 78 flop, plus 6 sine/cosine (MUFU, separate pipe).
FLOPS_PER_BIN_MIXED = 78
# The gradient adds per bin the combination of the three detectors' terms
# (3 x 4 FMA) and the basis-weighted sums (10 FMA): 22 FMA = 44 flop -> 122.
FLOPS_PER_BIN_GRAD = 122
# Calibration model (Section 2.2), per bin and detector on top of the plain
# likelihood: two spline values (4 FMA each, 16 flop), the phase shift (1),
# the amplitude factor (1 + 2) and the <h|h> correction (4): 24 flop.
FLOPS_PER_BIN_CAL = FLOPS_PER_BIN_MIXED + 3 * 24
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of one bin-loop launch on this workload, from the
# ncu capture summarised in profiles/k_window_mixed_c2.md; None whenever the
# kernel has changed since that capture.
KWINDOW_DRAM_BYTES = 1590272 + 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--soak-seconds", type=float, default=1.5)
    ap.add_argument("--impl", default="gwl", choices=["gwl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--shape", default="",
                    help="W,C: fixed likelihood launch shape (window bins, CTAs per SM) instead of the autotuner; "
                         "for profiler runs, whose timing would mislead the autotuner")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Seed of a replica's proposal batch: every rank evaluates its own proposals."""
    return SEED + 1000 * rank


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of per-rank timings over all ranks (the slowest replica sets the time)."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() \
            and torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units processed by all replicas per second, over the slowest replica's time per step."""
    return world * units_per_rank / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "window": "untimed soak of the same step + the timed steps"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def device_event(ctx, precision, name=None):
    """The benchmark event, with the injection made by the device library (no oracle on this leg)."""
    from paper_1909_11873_gb300 import gwl
    import torch

    cache = {}

    def zero_ctx(ev):
        key = id(ev.geom)
        if key not in cache:
            full = I.Sampling(np.arange(11, dtype=np.int32), np.zeros(11), np.zeros(11, dtype=np.int32),
                              np.zeros(11), np.ones(11), np.zeros(11, dtype=np.int32))
            cache[key] = gwl.Context(ev.freqs, np.zeros_like(ev.strain), ev.psd, ev.geom, gwl.GWL_FP64, ev.fcut_mode,
                                     ev.gmst, ev.t_ref, full)
        return cache[key]

    def waveform(ev, th):
        c = zero_ctx(ev)
        h = gwl.waveform(c, torch.from_numpy(np.ascontiguousarray(th[None])).cuda()).cpu().numpy()[0]
        return h[..., 0] + 1j * h[..., 1]

    def snr2(ev, th):
        c = zero_ctx(ev)
        return -2.0 * float(gwl.loglike(c, torch.from_numpy(np.ascontiguousarray(th[None])).cuda()).cpu()[0])

    ev = I.make_event(name or CONFIG, SEED, waveform, snr2)
    for c in cache.values():
        c.close()
    return ev


GRAD_BATCH = 4096
NS_K, NS_CHAINS, NS_WALK = 250, 250, 20


def in_band_pairs(ev, theta_full):
    """Sum over proposals of the in-band bin count (the ISCO cut from the proposal's total mass)."""
    eta = theta_full[:, 1] / (1 + theta_full[:, 1]) ** 2
    fisco = 1.0 / (6 ** 1.5 * math.pi * theta_full[:, 0] * eta ** -0.6 * 4.925490947e-6)
    return float(np.searchsorted(ev.freqs, fisco, side="right").sum())


def run_grad(ev, args, flush, stream, peak_tflops):
    """grad lnL evals/s on the same data (4096 proposals), device-timed, L2 flushed between steps."""
    import torch

    from paper_1909_11873_gb300 import gwl

    th = I.proposals(ev, GRAD_BATCH, SEED + 7)
    x = torch.from_numpy(I.reduced(th, ev.sampling)).cuda()
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    tuning = ctx.gwl_autotune(x, gwl.GWL_TUNE_GRAD, stream)
    out = torch.empty(GRAD_BATCH, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    for _ in range(args.warmup):
        ctx.gwl_grad(x, out, g, stream)
    torch.cuda.synchronize()
    steps = max(10, args.steps // 2)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        flush.fill_(1.0)
        e0.record(stream)
        ctx.gwl_grad(x, out, g, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    # the gradient bin loop's own time (library CUDA events on the launch stream)
    ctx.gwl_profile(True)
    for _ in range(steps):
        flush.fill_(1.0)
        ctx.gwl_grad(x, out, g, stream)
    torch.cuda.synchronize()
    kms, kn = ctx.gwl_profile_read(gwl.KERNEL_GRAD)
    ctx.gwl_profile(False)
    ctx.close()
    pairs = in_band_pairs(ev, th)
    achieved = FLOPS_PER_BIN_GRAD * pairs / (kms / kn * 1e-3) / 1e12
    return {"value": GRAD_BATCH / (ms * 1e-3), "unit": "grad evals/s", "ms_per_step": ms, "batch": GRAD_BATCH,
            "steps": steps, "precision": "mixed", "workload": "same 3-det 8 s data, 11-D gradient",
            "grad_window": tuning["grad_window"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "kernel": "k_window_grad<3,mixed>",
                         "flops_per_pair": FLOPS_PER_BIN_GRAD, "pairs_per_launch": int(pairs),
                         "kernel_ms": kms / kn}}


def run_cal(ev, args, flush, stream, peak_tflops):
    """lnL evals/s with the calibration model (ten amplitude and ten phase nodes per detector, 71 parameters
    per row) on the same data and batch, device-timed, L2 flushed between steps."""
    import torch

    from paper_1909_11873_gb300 import gwl

    th = I.calibrated_proposals(ev, BATCH, SEED + 11)
    rows = np.ascontiguousarray(np.concatenate([I.reduced(th[:, :11], ev.sampling), th[:, 11:]], axis=1))
    x = torch.from_numpy(rows).cuda()
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    ctx.gwl_set_calibration(I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1])))
    tuning = ctx.gwl_autotune(x, gwl.GWL_TUNE_LOGLIKE, stream)
    out = torch.empty(BATCH, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.gwl_loglike(x, out, stream)
    torch.cuda.synchronize()
    steps = max(10, args.steps // 2)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        flush.fill_(1.0)
        e0.record(stream)
        ctx.gwl_loglike(x, out, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    ctx.gwl_profile(True)
    for _ in range(steps):
        flush.fill_(1.0)
        ctx.gwl_loglike(x, out, stream)
    torch.cuda.synchronize()
    kms, kn = ctx.gwl_profile_read(gwl.KERNEL_BINS)
    ctx.gwl_profile(False)
    ctx.close()
    pairs = in_band_pairs(ev, th[:, :11])
    achieved = FLOPS_PER_BIN_CAL * pairs / (kms / kn * 1e-3) / 1e12
    return {"value": BATCH / (ms * 1e-3), "unit": "evals/s", "ms_per_step": ms, "batch": BATCH, "steps": steps,
            "precision": "mixed", "dim": int(rows.shape[1]),
            "workload": "same 3-det 8 s data, 11 source + 60 calibration parameters (10 nodes per detector)",
            "window": tuning["window"], "ctas_per_sm": tuning["ctas_per_sm"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "kernel": "k_window<3,mixed,calibrated>",
                         "flops_per_pair": FLOPS_PER_BIN_CAL, "pairs_per_launch": int(pairs),
                         "kernel_ms": kms / kn}}


def run_ns(args):
    """Wall time of a full nested-sampling run on the 1-detector 4 s zero-noise event (4-D)."""
    from paper_1909_11873_gb300 import gwl

    ev1 = device_event(None, None, name="c1")
    ctx = gwl.Context.from_event(ev1, gwl.GWL_MIXED)
    ctx.ns_run(NS_K, NS_CHAINS, NS_WALK, seed=1, dlogz=0.1, max_rounds=2)  # warm-up (graph build, scratch)
    t0 = time.perf_counter()
    r = ctx.ns_run(NS_K, NS_CHAINS, NS_WALK, seed=2, dlogz=0.1)
    wall = time.perf_counter() - t0
    ctx.close()
    return {"wall_s": wall, "lnZ": r["lnZ"], "lnZ_err": r["lnZ_err"], "rounds": r["rounds"],
            "n_proposals": r["n_proposals"], "consumed_per_round": r["consumed_per_round"],
            "workload": f"1-det 4 s 20-512 Hz zero-noise, 4-D, K={NS_K}, {NS_CHAINS} chains, walk {NS_WALK}, "
                        "dlogz 0.1, mixed precision"}


def run_gwl(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1909_11873_gb300 import build, gwl

    if not os.path.exists(gwl.LIB_PATH):
        build.build()
    ev = device_event(None, None)
    theta_full = I.proposals(ev, BATCH, rank_seed(rank))
    theta_np = np.ascontiguousarray(I.reduced(theta_full, ev.sampling))
    theta = torch.from_numpy(theta_np).cuda()
    lnl = torch.empty(BATCH, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(ctx, steps, warmup, host=False, soak=0.0, nvtx=None):
        # pinned host buffers, as a caller would hold them (numpy views made once)
        host_t = torch.from_numpy(theta_np).pin_memory().numpy() if host else None
        host_l = torch.empty(BATCH, dtype=torch.float64).pin_memory().numpy() if host else None
        for _ in range(warmup):
            if host:
                ctx.gwl_loglike_host(host_t, host_l, stream)
            else:
                ctx.gwl_loglike(theta, lnl, stream)
        torch.cuda.synchronize()
        # untimed soak at load so that the clock sampler sees the GPU under this workload
        t_end = time.perf_counter() + soak
        while time.perf_counter() < t_end:
            for _ in range(50):
                flush.fill_(1.0)
                ctx.gwl_loglike(theta, lnl, stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        l0 = ctx.launch_count()
        # an NVTX range around the timed steps lets a profiler list exactly these launches
        rng = torch.cuda.nvtx.range_start(nvtx) if nvtx else None
        wall0 = time.perf_counter()
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            if host:
                ctx.gwl_loglike_host(host_t, host_l, stream)
            else:
                ctx.gwl_loglike(theta, lnl, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if rng is not None:
            torch.cuda.nvtx.range_end(rng)
        if world > 1:
            torch.distributed.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return sum(ms) / len(ms), ctx.launch_count() - l0, wall

    results = {}
    ctxs = {}
    tuning = {}
    for prec in (gwl.GWL_FP64, gwl.GWL_MIXED):
        ctx = gwl.Context.from_event(ev, prec)
        ctxs[prec] = ctx
        # launch shape from the library's autotuner on this batch (untimed), or fixed by --shape
        if args.shape and prec == gwl.GWL_MIXED:
            w, c = (int(v) for v in args.shape.split(","))
            ctx.gwl_set_tuning(window=w, ctas_per_sm=c)
            tuning["mixed"] = dict(ctx.gwl_get_tuning(), fixed=True)
        else:
            tuning["mixed" if prec == gwl.GWL_MIXED else "fp64"] = ctx.gwl_autotune(theta, gwl.GWL_TUNE_LOGLIKE,
                                                                                    stream)
        steps = args.steps if prec == gwl.GWL_MIXED else max(3, args.steps // 5)
        with ClockSampler(local) as clk:
            ms, launches, wall = timed(ctx, steps, args.warmup, soak=args.soak_seconds,
                                       nvtx="timed_mixed" if prec == gwl.GWL_MIXED else "timed_fp64")
        ctx.gwl_sync()
        results[prec] = dict(ms=ms, launches=launches, clocks=clk.summary(), steps=steps, wall=wall)

    mixed = ctxs[gwl.GWL_MIXED]
    # dominant kernel timing (library CUDA events on the launch stream) over a separate timed pass
    mixed.gwl_profile(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        mixed.gwl_loglike(theta, lnl, stream)
    torch.cuda.synchronize()
    prof = {k: mixed.gwl_profile_read(k) for k in (gwl.KERNEL_PROLOGUE, gwl.KERNEL_BINS, gwl.KERNEL_COMBINE)}
    mixed.gwl_profile(False)

    # end-to-end with host buffers
    ms_e2e, _, _ = timed(mixed, max(5, args.steps // 2), args.warmup, host=True)
    # algorithmic work of one launch: in-band (proposal, bin) pairs (ncut from the prologue's f_ISCO)
    pairs = in_band_pairs(ev, theta_full)
    # the bin loop of one call (one launch; it also forms lnL)
    bins_ms, bins_n = prof[gwl.KERNEL_BINS]
    per_launch_s = bins_ms / args.steps * 1e-3
    peaks = measured_peaks()
    clk = results[gwl.GWL_MIXED]["clocks"]
    fclk = (clk["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    import torch as _t
    n_sm = _t.cuda.get_device_properties(local).multi_processor_count
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * fclk / 1e12
    achieved = FLOPS_PER_BIN_MIXED * pairs / per_launch_s / 1e12
    grad_res = run_grad(ev, args, flush, stream, peak_tflops) if rank == 0 else None
    cal_res = run_cal(ev, args, flush, stream, peak_tflops) if rank == 0 else None
    ns_res = run_ns(args) if rank == 0 else None

    ms, ms64, mse = max_over_ranks([results[gwl.GWL_MIXED]["ms"], results[gwl.GWL_FP64]["ms"], ms_e2e], "cuda")
    value = whole_job_rate(BATCH, world, ms)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32x2-phase/f32/f64",
        "data": "synthetic (seeded coloured Gaussian noise + TaylorF2 injection from the device template)",
        "config": {"workload": "3-det BBH, 8 s, 20-1024 Hz, 8033 bins/det, 11-D, batch 8192 proposals per GPU",
                   "global_batch": BATCH * world, "bins_per_det": int(ev.M), "n_det": int(ev.n_det),
                   "in_band_pairs_per_batch": int(pairs), "precision": "mixed",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "fp64_path": {"value": whole_job_rate(BATCH, world, ms64), "ms_per_step": ms64, "steps": results[gwl.GWL_FP64]["steps"],
                      "speedup_mixed_over_fp64": ms64 / ms},
        "e2e": {"value": whole_job_rate(BATCH, world, mse), "unit": "evals/s", "h2d_bytes_per_step": int(theta_np.nbytes),
                "d2h_bytes_per_step": int(BATCH * 8)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": KWINDOW_DRAM_BYTES,
                     "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_window<3,mixed> "
                                      "launch (704-bin windows, 2 CTAs/SM; profiles/k_window_mixed_c2.md)",
                     "kernel": "k_window<3,mixed> (windowed bin loop and lnL combination)",
                     "peak_basis": f"FP32 pipe: {n_sm} SMs x 128 lanes x 2 flop x {fclk / 1e6:.0f} MHz (derived)",
                     "flops_per_pair": FLOPS_PER_BIN_MIXED, "pairs_per_launch": int(pairs),
                     "kernel_ms": per_launch_s * 1e3,
                     "share_of_step": bins_ms / args.steps / ms},
        "kernel_ms": {"prologue": prof[gwl.KERNEL_PROLOGUE][0] / args.steps,
                      "bins": bins_ms / args.steps,
                      "combine": prof[gwl.KERNEL_COMBINE][0] / args.steps},
        "tuning": {k: {f: v[f] for f in ("window", "ctas_per_sm", "ms_loglike", "n_tried")}
                   for k, v in tuning.items()},
        "clocks": clk,
        "gpu_launches": int(results[gwl.GWL_MIXED]["launches"]),
        "grad": grad_res,
        "calibrated": cal_res,
        "ns": ns_res,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(theta_full, args.cpu_seconds, use_device_event=ev)
        out["accuracy"] = out["cpu_baseline"].pop("accuracy")
        out["cpu_baseline"]["ns_wall_s"] = oracle_ns_wall()
    for c in ctxs.values():
        c.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_event():
    import oracle

    def wf(ev, th):
        return oracle.waveform(ev, th)

    def snr2(ev, th):
        return -2.0 * oracle.loglike(ev.with_strain(np.zeros_like(ev.strain)), th[None])[0]

    return I.make_event(CONFIG, SEED, wf, snr2)


def cpu_baseline(theta_full, seconds, use_device_event=None):
    """The FP64 oracle (as it stands) on all host cores, repeated over the batch until ~seconds elapse."""
    import oracle

    ev = oracle_event()
    n = os.cpu_count() or 1
    sample = theta_full[:1024]
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.loglike(ev, sample, n_threads=n)
        done += sample.shape[0]
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "evals/s", "cores": n, "kind": "oracle",
            "sample": f"{done} evaluations = repeated first 1024 proposals of the 8192-proposal batch "
                      f"(same event, oracle-made injection), {el:.1f} s wall",
            "accuracy": device_accuracy(ev, sample, oracle.loglike(ev, sample, n_threads=n))}


def device_accuracy(ev, theta_full, ref):
    """max |lnL_device - lnL_oracle| of both device paths on the oracle's own event (bars 1e-6 / 1e-3)."""
    import torch

    from paper_1909_11873_gb300 import gwl

    x = torch.from_numpy(np.ascontiguousarray(I.reduced(theta_full, ev.sampling))).cuda()
    out = {"rows": int(theta_full.shape[0]), "max_abs_lnL": float(np.max(np.abs(ref)))}
    for name, prec in (("fp64", gwl.GWL_FP64), ("mixed", gwl.GWL_MIXED)):
        ctx = gwl.Context.from_event(ev, prec)
        got = gwl.loglike(ctx, x).cpu().numpy()
        ctx.gwl_sync()
        ctx.close()
        out[f"{name}_max_abs_err"] = float(np.max(np.abs(got - ref)))
    out["bars"] = {"fp64": 1e-6, "mixed": 1e-3}
    return out


def oracle_ns_wall():
    """The oracle's nested sampler on the same 1-detector event and settings (host cores)."""
    import oracle

    def wf(ev, th):
        return oracle.waveform(ev, th)

    def snr2(ev, th):
        return -2.0 * oracle.loglike(ev.with_strain(np.zeros_like(ev.strain)), th[None])[0]

    ev1 = I.make_event("c1", SEED, wf, snr2)
    t0 = time.perf_counter()
    r = oracle.ns_run(ev1, ev1.sampling, NS_K, NS_CHAINS, NS_WALK, seed=2, dlogz=0.1)
    return {"wall_s": time.perf_counter() - t0, "lnZ": r["lnZ"], "lnZ_err": r["lnZ_err"], "rounds": r["rounds"],
            "cores": os.cpu_count()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    ev = oracle_event()
    theta_full = I.proposals(ev, BATCH, SEED)
    n = os.cpu_count() or 1
    sample = theta_full[:512]
    for _ in range(args.warmup):
        oracle.loglike(ev, sample[:64], n_threads=n)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.loglike(ev, sample, n_threads=n)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * sum(ts) / len(ts)
    value = sample.shape[0] / (ms * 1e-3)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "3-det BBH, 8 s, 20-1024 Hz, 8033 bins/det, 11-D; each step 512 of the 8192 proposals",
                   "global_batch": BATCH, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": n, "kind": "oracle",
                         "sample": "512 proposals of the 8192-proposal batch per step"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gwl(args)


if __name__ == "__main__":
    main()
