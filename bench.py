#!/usr/bin/env python3
"""Benchmark: batched TaylorF2 lnL evaluations per second on one GB300 (or N, weak scaling).

Workload (one step): one gwl_loglike call over a batch of 8192 proposals for
a 3-detector, 8 s, 20-1024 Hz network (8033 bins per detector, coloured
Gaussian noise, 11-D aligned-spin BBH injection at SNR 15-30); half the
proposals are prior draws and half perturb the injection.  Inputs are
synthetic and seeded; the injections are produced by the device library's
own template (gwl_waveform), so the GPU legs run no oracle code.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gwl|reference] [--legs a,b,...]

Prints one JSON line (rank 0).  ``value`` is the mixed-precision path's
device-timed throughput with inputs resident in HBM; L2 (129 MB) is flushed
by writing a 256 MB buffer between timed steps (the step inputs are < 1 MB).
``e2e`` is the same metric through gwl_loglike_host with page-locked host
buffers, timed by the host clock around each call (the flush is issued and
finished before the clock starts).  ``roofline`` refers to the dominant
kernel (the windowed bin loop), timed by the library's CUDA events on the
launch stream, with every pipe's algorithmic work reported and the largest
fraction taken as the bound.  ``cpu_baseline`` times the FP64 oracle on the
host cores on a bounded sample and runs the oracle comparisons of the other
legs.  The other measurements come last in the line, compactly, under
``legs``: the plain FP64 path, the FP64-phase mixed arm, the gradient, the
calibrated likelihood, the 1-detector and 128 s workloads, the 64-event
workload, the two walks' effective samples per second and a full nested
sampling run.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
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
LEGS = ("fp64", "fp64ph", "grad", "cal", "calgrad", "c1", "c3", "c4", "c5", "ns")

# Algorithmic work of the mixed likelihood bin loop per in-band (proposal, bin)
# pair with 3 detectors, counted from the arithmetic the kernel carries out
# for that pair (FMA = 2 flop; TwoProduct = 3, TwoSum = 6):
#   FP32: the phase delta sum_m c_m dB_m over 8 basis terms (15), its nearest
#     integer and subtraction (3); per detector the anchor-plus-lane term (1),
#     the sum with the delta (1), the scaling to radians (1) and the four
#     multiply-adds of U and V (8): 3 x 11 = 33; the block's float-float anchor
#     term (about 180 flop per 32-bin block) -> 5: 56 flop.
#   MUFU (special-function unit): sine and cosine per detector -> 6.
#   FP64: the combination, about 40 flop per proposal (not per pair) -> 0.
#   HBM: theta in (88 B) and lnL out (8 B) per proposal.
PIPES_MIXED = {"fp32_flop": 56, "mufu": 6}
HBM_BYTES_PER_EVAL = 96
# The gradient bin loop per pair: the exact float-float phase per bin (the
# 8-term sum, pairwise: 8 TwoProducts, 7 TwoSums and the low-part terms, 114;
# per detector the delay term, TwoSum and reduction, 3 x 20) -> 174; per
# detector the sine and cosine of the reduced phase from a table of the
# 64th-cycle points and short series on the FP32 pipe (reduction 5, scaling
# 1, the two series 8, the rotation 6: 20) -> 60; per
# detector the data-weighted phasor (6), Z_d (2), the imaginary part of K_d
# times it (3), its f-weighted sum (2) and the sum over detectors (1) ->
# 3 x 14 = 42; the eight basis-weighted sums of that total (16): 292 flop;
# no MUFU.
PIPES_GRAD = {"fp32_flop": 292, "mufu": 0}
# Calibration model (Section 2.2), per bin on top of the plain likelihood: the
# four spline weights (9 flop, shared by the detectors); per detector two
# spline values (2 x 7), the phase shift (1), the amplitude factor (3) and the
# <h|h> correction (4): 9 + 3 x 22 = 75.
PIPES_CAL = {"fp32_flop": 56 + 75, "mufu": 6}
FP32_LANES_PER_SM = 128
MUFU_PER_SM_CLK = 16
# The kernel sources whose change invalidates a stored DRAM-traffic capture.
KERNEL_SOURCES = ("gwl_lnl.cu", "gwl_bins.cuh", "gwl_sched.cuh", "gwl_device.cuh", "gwl_ff.cuh", "gwl_internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_k_window_mixed_c2.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--soak-seconds", type=float, default=1.5)
    ap.add_argument("--impl", default="gwl", choices=["gwl", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--legs", default=",".join(LEGS), help="extra measurements to run (comma list; '' for none)")
    ap.add_argument("--profile-only", default="",
                    choices=["", "lnl", "grad", "cal", "calgrad", "fp64ph", "fp64", "ns"],
                    help="run one workload --warmup + --steps times without timing and exit (for profiler captures): "
                         "lnl = the headline likelihood, grad = the 4096-proposal gradient, cal = the calibrated "
                         "likelihood, fp64ph = the FP64-phase mixed arm")
    ap.add_argument("--profile-config", default="c2", choices=["c2", "c3"],
                    help="--profile-only workload: c2 = the 3-detector 8 s batch, c3 = the 128 s BNS batch (2048)")
    ap.add_argument("--bin-kernel", type=int, default=0, choices=[0, 1, 2, 3],
                    help="likelihood bin-loop layout for --shape / --profile-only runs (1 auto, 2 warp, 3 lane)")
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


def r4(x):
    """A number rounded to four significant digits (compact JSON)."""
    if x is None:
        return None
    if isinstance(x, (list, tuple)):
        return [r4(v) for v in x]
    if isinstance(x, dict):
        return {k: r4(v) for k, v in x.items()}
    if isinstance(x, (bool, str)):
        return x
    if isinstance(x, (int, np.integer)):
        return int(x)
    x = float(x)
    return x if x == 0.0 or not math.isfinite(x) else float(f"{x:.4g}")


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


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1909_11873_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stored_traffic():
    """DRAM bytes of one bin-loop launch from the committed one-pass ncu capture, or None when the
    kernel sources have changed since that capture (its source hash no longer matches)."""
    try:
        kv = dict(ln.split(":", 1) for ln in open(TRAFFIC_FILE).read().splitlines() if ":" in ln)
    except OSError:
        return None, "no capture"
    if kv.get("kernel_source_sha16", "").strip() != kernel_source_hash():
        return None, "kernel changed since the capture"
    return int(kv["dram_bytes_per_launch"].strip()), "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"


def device_event(name=None, seed=SEED, cfg=None, fcut_mode=0):
    """A synthetic event whose injection comes from the device library's own template (no oracle)."""
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

    ev = I.make_event(name or "custom", seed, waveform, snr2, cfg=cfg, fcut_mode=fcut_mode)
    for c in cache.values():
        c.close()
    return ev


def in_band_pairs(ev, theta_full):
    """Sum over proposals of the in-band bin count (the ISCO cut from the proposal's total mass)."""
    eta = theta_full[:, 1] / (1 + theta_full[:, 1]) ** 2
    fisco = 1.0 / (6 ** 1.5 * math.pi * theta_full[:, 0] * eta ** -0.6 * 4.925490947e-6)
    return float(np.searchsorted(ev.freqs, fisco, side="right").sum())


def pipe_roofline(pipes, pairs, kernel_ms, n_sm, fclk, n_eval):
    """Every pipe's achieved rate against its derived peak; the bound is the largest fraction."""
    s = kernel_ms * 1e-3
    peaks = {"fp32_flop": n_sm * FP32_LANES_PER_SM * 2 * fclk, "mufu": n_sm * MUFU_PER_SM_CLK * fclk}
    out = {}
    for k, per_pair in pipes.items():
        a = per_pair * pairs / s
        out[k] = {"per_pair": per_pair, "achieved_T": a / 1e12, "peak_T": peaks[k] / 1e12, "frac": a / peaks[k]}
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    a = HBM_BYTES_PER_EVAL * n_eval / s / 1e9
    out["hbm"] = {"per_eval_bytes": HBM_BYTES_PER_EVAL, "achieved_GBs": a, "peak_GBs": hbm, "frac": a / hbm}
    bound = max(out, key=lambda k: out[k]["frac"])
    return bound, out


def time_device(fn, steps, flush, stream):
    """Mean device time (ms) of fn() over `steps` calls, CUDA events on the launch stream, L2 flushed before each."""
    import torch

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        flush.fill_(1.0)
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


# ---------------------------------------------------------------- extra legs (rank 0)
def leg_grad(ev, args, flush, stream, n_sm, fclk):
    """grad lnL evals/s on the same data (4096 proposals), device-timed, L2 flushed between steps."""
    import torch

    from paper_1909_11873_gb300 import gwl

    B = 4096
    th = I.proposals(ev, B, SEED + 7)
    x = torch.from_numpy(I.reduced(th, ev.sampling)).cuda()
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    tuning = ctx.gwl_autotune(x, gwl.GWL_TUNE_GRAD, stream)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    for _ in range(args.warmup):
        ctx.gwl_grad(x, out, g, stream)
    torch.cuda.synchronize()
    steps = max(10, args.steps // 2)
    ms = time_device(lambda: ctx.gwl_grad(x, out, g, stream), steps, flush, stream)
    ctx.gwl_profile(True)
    for _ in range(steps):
        flush.fill_(1.0)
        ctx.gwl_grad(x, out, g, stream)
    torch.cuda.synchronize()
    kms, kn = ctx.gwl_profile_read(gwl.KERNEL_GRAD)
    ctx.gwl_profile(False)
    ctx.gwl_sync()
    ctx.close()
    bound, pipes = pipe_roofline(PIPES_GRAD, in_band_pairs(ev, th), kms / kn, n_sm, fclk, B)
    return {"v": B / (ms * 1e-3), "ms": ms, "B": B, "win": tuning["grad_window"], "kernel_ms": kms / kn,
            "bound": bound, "frac": pipes[bound]["frac"], "fp32_frac": pipes["fp32_flop"]["frac"]}


def leg_calgrad(ev, args, flush, stream):
    """grad lnL evals/s with the calibration model (71 parameters per row: the gradient's row is the same
    size) on 4096 proposals of the same data; device time per call and the two bin passes' kernel times."""
    import torch

    from paper_1909_11873_gb300 import gwl

    B = 4096
    th = I.calibrated_proposals(ev, B, SEED + 13)
    rows = np.ascontiguousarray(np.concatenate([I.reduced(th[:, :11], ev.sampling), th[:, 11:]], axis=1))
    x = torch.from_numpy(rows).cuda()
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    ctx.gwl_set_calibration(I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1])))
    tuning = ctx.gwl_autotune(x, gwl.GWL_TUNE_GRAD, stream)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    for _ in range(args.warmup):
        ctx.gwl_grad(x, out, g, stream)
    torch.cuda.synchronize()
    steps = max(10, args.steps // 2)
    ms = time_device(lambda: ctx.gwl_grad(x, out, g, stream), steps, flush, stream)
    ctx.gwl_profile(True)
    for _ in range(steps):
        flush.fill_(1.0)
        ctx.gwl_grad(x, out, g, stream)
    torch.cuda.synchronize()
    gms, gn = ctx.gwl_profile_read(gwl.KERNEL_GRAD)
    cms, cn = ctx.gwl_profile_read(gwl.KERNEL_CALGRAD)
    ctx.gwl_profile(False)
    ctx.gwl_sync()
    ctx.close()
    return {"v": B / (ms * 1e-3), "ms": ms, "dim": int(rows.shape[1]), "win": tuning["grad_window"],
            "grad_bins_ms": gms / max(gn, 1), "cal_moments_ms": cms / max(cn, 1)}


def leg_cal(ev, args, flush, stream, n_sm, fclk):
    """lnL evals/s with the calibration model (ten amplitude and ten phase nodes per detector, 71 parameters
    per row) on the same data and batch size."""
    import torch

    from paper_1909_11873_gb300 import gwl

    th = I.calibrated_proposals(ev, BATCH, SEED + 11)
    rows = np.ascontiguousarray(np.concatenate([I.reduced(th[:, :11], ev.sampling), th[:, 11:]], axis=1))
    x = torch.from_numpy(rows).cuda()
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    ctx.gwl_set_calibration(I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1])))
    ctx.gwl_autotune(x, gwl.GWL_TUNE_LOGLIKE, stream)
    out = torch.empty(BATCH, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.gwl_loglike(x, out, stream)
    torch.cuda.synchronize()
    steps = max(10, args.steps // 2)
    ms = time_device(lambda: ctx.gwl_loglike(x, out, stream), steps, flush, stream)
    ctx.gwl_profile(True)
    for _ in range(steps):
        flush.fill_(1.0)
        ctx.gwl_loglike(x, out, stream)
    torch.cuda.synchronize()
    kms, kn = ctx.gwl_profile_read(gwl.KERNEL_BINS)
    ctx.gwl_profile(False)
    ctx.gwl_sync()
    ctx.close()
    bound, pipes = pipe_roofline(PIPES_CAL, in_band_pairs(ev, th[:, :11]), kms / kn, n_sm, fclk, BATCH)
    return {"v": BATCH / (ms * 1e-3), "ms": ms, "dim": int(rows.shape[1]), "kernel_ms": kms / kn, "bound": bound,
            "frac": pipes[bound]["frac"]}


def lnl_rates(ev, B, seed, args, flush, stream, precisions, local_fraction=0.5, tune=True):
    """Device-timed lnL evals/s of each precision mode on one event and batch."""
    import torch

    from paper_1909_11873_gb300 import gwl

    th = I.proposals(ev, B, seed, local_fraction=local_fraction)
    x = torch.from_numpy(I.reduced(th, ev.sampling)).cuda()
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    res = {}
    for name, prec in precisions:
        ctx = gwl.Context.from_event(ev, prec)
        if tune and prec != gwl.GWL_FP64:
            ctx.gwl_autotune(x, gwl.GWL_TUNE_LOGLIKE, stream)
        ctx.gwl_loglike(x, out, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.gwl_loglike(x, out, stream)
        torch.cuda.synchronize()
        one = time.perf_counter() - t0
        steps = int(min(max(3, args.steps // 4), max(3, 1.0 / max(one, 1e-6))))
        ms = time_device(lambda: ctx.gwl_loglike(x, out, stream), steps, flush, stream)
        ctx.gwl_sync()
        ctx.close()
        res[name] = B / (ms * 1e-3)
    return res


def four_d(ev):
    """The event with (Mc, q, tc, phic) sampled in narrow priors around the injection, the other parameters at
    the injection: a unimodal posterior on which lnZ comparisons are well posed."""
    th = ev.theta_inj
    bns = th[0] < 5
    smp = I.Sampling(np.array([0, 1, 9, 10], dtype=np.int32), th.copy(), np.zeros(4, dtype=np.int32),
                     np.array([th[0] * (0.995 if bns else 0.97), 0.7 if bns else 0.25, -0.02, 0.0]),
                     np.array([th[0] * (1.005 if bns else 1.03), 1.0, 0.02, 2 * math.pi]),
                     np.array([0, 0, 0, 1], dtype=np.int32))
    return dataclasses.replace(ev, sampling=smp)


C4_K, C4_CHAINS, C4_WALK, C4_SEED = 1000, 1000, 100, 4


def leg_c4(args, flush, stream):
    """64 events of {4..128} s (3 detectors, 20-1024 Hz, BBH or BNS): one batched lnL call over 1000
    proposals per event vs per-event calls, and full nested-sampling runs of all events (K = 1000,
    1000 chains, walk 100, 4-D sampling) as one graph per round vs 64 per-event ns_run calls."""
    import torch

    from paper_1909_11873_gb300 import gwl

    cfgs = I.c4_events(C4_SEED, 64)
    evs = [four_d(device_event(cfg=c, seed=c["seed"])) for c in cfgs]
    ths = [I.proposals(ev, C4_K, c["seed"]) for ev, c in zip(evs, cfgs)]
    ctxs = [gwl.Context.from_event(ev, gwl.GWL_MIXED) for ev in evs]
    mc = gwl.MultiContext(ctxs)
    x = torch.from_numpy(np.concatenate([I.reduced(t, ev.sampling) for t, ev in zip(ths, evs)])).cuda()
    xs = [x[i * C4_K:(i + 1) * C4_K] for i in range(len(evs))]
    out = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
    outs = [torch.empty(C4_K, dtype=torch.float64, device="cuda") for _ in evs]
    mc.gwl_multi_loglike(x, out)
    [c.gwl_loglike(xx, o) for c, xx, o in zip(ctxs, xs, outs)]
    torch.cuda.synchronize()
    ms_b = time_device(lambda: mc.gwl_multi_loglike(x, out, stream), 5, flush, stream)
    ms_e = time_device(lambda: [c.gwl_loglike(xx, o, stream) for c, xx, o in zip(ctxs, xs, outs)], 5, flush, stream)
    diff = float((torch.cat(outs) - out).abs().max())
    # nested sampling: all events in one graph per round, then event by event
    mc.gwl_multi_ns_run(C4_K, C4_CHAINS, C4_WALK, seed=1, dlogz=0.1, max_rounds=1)  # warm-up
    t0 = time.perf_counter()
    rb = mc.gwl_multi_ns_run(C4_K, C4_CHAINS, C4_WALK, seed=C4_SEED, dlogz=0.1)
    wall_b = time.perf_counter() - t0
    ctxs[0].ns_run(C4_K, C4_CHAINS, C4_WALK, seed=1, dlogz=0.1, max_rounds=1)  # warm-up
    t0 = time.perf_counter()
    re = [c.ns_run(C4_K, C4_CHAINS, C4_WALK, seed=C4_SEED + 1 + e, dlogz=0.1) for e, c in enumerate(ctxs)]
    wall_e = time.perf_counter() - t0
    z = np.array([[a["lnZ"] - b["lnZ"], math.hypot(a["lnZ_err"], b["lnZ_err"])] for a, b in zip(rb, re)])
    mc.close()
    for c in ctxs:
        c.close()
    return {"lnl_batched_ms": ms_b, "lnl_per_event_ms": ms_e, "lnl_x": ms_e / ms_b, "lnl_diff": diff,
            "ns_graph_s": wall_b, "ns_per_event_s": wall_e, "ns_x": wall_e / wall_b,
            "rounds": int(max(r["rounds"] for r in rb)),
            "lnZ_graph_vs_per_event_max_sigma": float(np.max(np.abs(z[:, 0]) / z[:, 1])),
            "durations": sorted({int(c["T"]) for c in cfgs})}


def leg_c5(ev, args):
    """Random walk vs gradient-informed (Galilean) walk inside nested sampling on the 3-detector 8 s event:
    Kish effective samples per second over three seeds, in 4-D and 11-D (K = 500, walk 20)."""
    from paper_1909_11873_gb300 import gwl

    out = {}
    for dims in (4, 11):
        e = four_d(ev) if dims == 4 else ev
        row = {}
        for name, kind in (("random", gwl.GWL_WALK_RANDOM), ("galilean", gwl.GWL_WALK_GALILEAN)):
            ctx = gwl.Context.from_event(e, gwl.GWL_MIXED)
            ctx.gwl_set_walk(kind)
            ctx.ns_run(500, 500, 20, seed=999, dlogz=0.1, max_rounds=1)  # warm-up
            ess, lnz = [], []
            for sd in range(3):
                t0 = time.perf_counter()
                r = ctx.ns_run(500, 500, 20, seed=100 + sd, dlogz=0.1, max_dead=400000)
                wall = time.perf_counter() - t0
                lw = r["dead_lnl"] + r["dead_logwt"]
                w = np.exp(lw - lw.max())
                ess.append(w.sum() ** 2 / (w ** 2).sum() / wall)
                lnz.append(r["lnZ"])
            ctx.close()
            row[name] = {"ess_s": float(np.mean(ess)), "lnZ": float(np.mean(lnz)), "spread": float(np.std(lnz, ddof=1))}
        out[f"{dims}d"] = row
    return out


NS_K, NS_CHAINS, NS_WALK = 250, 250, 20


def leg_ns():
    """Wall time of a full nested-sampling run on the 1-detector 4 s zero-noise event (4-D)."""
    from paper_1909_11873_gb300 import gwl

    ev1 = device_event("c1")
    ctx = gwl.Context.from_event(ev1, gwl.GWL_MIXED)
    ctx.ns_run(NS_K, NS_CHAINS, NS_WALK, seed=1, dlogz=0.1, max_rounds=2)  # warm-up (graph build, scratch)
    t0 = time.perf_counter()
    r = ctx.ns_run(NS_K, NS_CHAINS, NS_WALK, seed=2, dlogz=0.1)
    wall = time.perf_counter() - t0
    ctx.close()
    return {"wall_s": wall, "lnZ": r["lnZ"], "lnZ_err": r["lnZ_err"], "rounds": r["rounds"],
            "consumed": r["consumed_per_round"], "eq5": NS_K * math.log(1 + NS_CHAINS / NS_K)}


def leg_eq5():
    """Candidates consumed per round against Eq. 5's K ln(1 + B/K), and the run's wall time, for several
    batch sizes B at K = 250 (1-detector 4 s event, walk 20): the device analogue of the paper's Fig. 1."""
    from paper_1909_11873_gb300 import gwl

    ev1 = device_event("c1")
    ctx = gwl.Context.from_event(ev1, gwl.GWL_MIXED)
    ctx.ns_run(NS_K, 64, NS_WALK, seed=99, dlogz=0.1, max_rounds=2)  # warm-up
    rows = []
    for B in (25, 250, 1000, 4000):
        t0 = time.perf_counter()
        r = ctx.ns_run(NS_K, B, NS_WALK, seed=1000 + B, dlogz=0.1)
        wall = time.perf_counter() - t0
        rows.append([B, r["consumed_per_round"] / (NS_K * math.log(1 + B / NS_K)), int(r["rounds"]), wall])
    ctx.close()
    return {"cols": ["B", "consumed/eq5", "rounds", "wall_s"], "rows": rows}


# ---------------------------------------------------------------- main leg
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
    legs = [x for x in args.legs.split(",") if x] if rank == 0 else []
    ev = device_event(CONFIG)
    theta_full = I.proposals(ev, BATCH, rank_seed(rank))
    theta_np = np.ascontiguousarray(I.reduced(theta_full, ev.sampling))
    theta = torch.from_numpy(theta_np).cuda()
    lnl = torch.empty(BATCH, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(ctx, steps, warmup, soak=0.0, nvtx=None):
        for _ in range(warmup):
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
        l0 = ctx.launch_count()
        # an NVTX range around the timed steps lets a profiler list exactly these launches
        rng = torch.cuda.nvtx.range_start(nvtx) if nvtx else None
        ms = time_device(lambda: ctx.gwl_loglike(theta, lnl, stream), steps, flush, stream)
        if rng is not None:
            torch.cuda.nvtx.range_end(rng)
        if world > 1:
            torch.distributed.barrier()
        return ms, ctx.launch_count() - l0

    def timed_host(ctx, steps, warmup):
        """End to end through the public host-buffer entry point: the host clock around each call (the call
        synchronises before returning); the flush is issued and finished before the clock starts."""
        host_t = torch.from_numpy(theta_np).pin_memory().numpy()
        host_l = torch.empty(BATCH, dtype=torch.float64).pin_memory().numpy()
        for _ in range(warmup):
            ctx.gwl_loglike_host(host_t, host_l, stream)
        if world > 1:
            torch.distributed.barrier()
        walls = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.gwl_loglike_host(host_t, host_l, stream)
            walls.append(time.perf_counter() - t0)
        if world > 1:
            torch.distributed.barrier()
        # the same calls bracketed by CUDA events instead (the host's submission and return fall outside)
        dev = time_device(lambda: ctx.gwl_loglike_host(host_t, host_l, stream), steps, flush, stream)
        return 1e3 * sum(walls) / len(walls), dev

    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    if args.shape:
        w, c = (int(v) for v in args.shape.split(","))
        ctx.gwl_set_tuning(window=w, ctas_per_sm=c, bin_kernel=args.bin_kernel)
        tuning = dict(ctx.gwl_get_tuning(), fixed=True)
    else:
        tuning = ctx.gwl_autotune(theta, gwl.GWL_TUNE_LOGLIKE, stream)
    with ClockSampler(local) as clk:
        ms, launches = timed(ctx, args.steps, args.warmup, soak=args.soak_seconds, nvtx="timed_mixed")
    ctx.gwl_sync()
    clocks = clk.summary()
    # the bin loop's own time (library CUDA events on the launch stream) over a separate pass
    ctx.gwl_profile(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        ctx.gwl_loglike(theta, lnl, stream)
    torch.cuda.synchronize()
    prof = {k: ctx.gwl_profile_read(k) for k in (gwl.KERNEL_PROLOGUE, gwl.KERNEL_BINS)}
    ctx.gwl_profile(False)
    ms_host, ms_host_dev = timed_host(ctx, max(5, args.steps // 2), args.warmup)
    ctx.gwl_sync()

    pairs = in_band_pairs(ev, theta_full)
    bins_ms = prof[gwl.KERNEL_BINS][0] / args.steps
    peaks = measured_peaks()
    fclk = (clocks["sm_max_mhz"] or peaks.get("sm_max_mhz", 2070.0)) * 1e6
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    bound, pipes = pipe_roofline(PIPES_MIXED, pairs, bins_ms, n_sm, fclk, BATCH)
    traffic, traffic_basis = stored_traffic()

    ms, mse = max_over_ranks([ms, ms_host], "cuda")
    value = whole_job_rate(BATCH, world, ms)
    b = pipes[bound]
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
                   "global_batch": BATCH * world, "in_band_pairs_per_batch": int(pairs), "precision": "mixed",
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "window": tuning["window"], "ctas_per_sm": tuning["ctas_per_sm"],
                   "bin_kernel": {1: "auto", 2: "warp", 3: "lane"}.get(tuning.get("bin_kernel"), "?")},
        "e2e": {"value": whole_job_rate(BATCH, world, mse), "unit": "evals/s", "ms_per_call_host_clock": mse,
                "device_events_value": whole_job_rate(BATCH, world, ms_host_dev),
                "h2d_bytes_per_step": int(theta_np.nbytes), "d2h_bytes_per_step": int(BATCH * 8)},
        "roofline": {"bound": "alu", "pipe": bound, "achieved": b.get("achieved_T"), "peak": b.get("peak_T"),
                     "unit": "Top/s" if bound == "mufu" else "TFLOP/s", "frac": b["frac"], "traffic": traffic,
                     "traffic_basis": traffic_basis,
                     "kernel": "k_lanes<3>" if tuning.get("bin_kernel") == 3 else "k_window<3,mixed>", "kernel_ms": bins_ms,
                     "pairs_per_launch": int(pairs), "share_of_step": bins_ms / ms,
                     "pipes": r4({k: {"per": v.get("per_pair", v.get("per_eval_bytes")), "frac": v["frac"]}
                                  for k, v in pipes.items()}),
                     "peak_basis": f"derived: {n_sm} SMs x {fclk / 1e6:.0f} MHz x (128 FP32 lanes x 2 | 16 MUFU)"},
        "kernel_ms": r4({"prologue": prof[gwl.KERNEL_PROLOGUE][0] / args.steps, "bins": bins_ms}),
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    ctx.close()
    legres = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(theta_full, args.cpu_seconds, legs)
    # extra measurements, compact, at the end of the line
    if "fp64" in legs:
        r = lnl_rates(ev, BATCH, rank_seed(rank), args, flush, stream, (("fp64", gwl.GWL_FP64),))
        legres["fp64_c2"] = {"v": r["fp64"], "mixed_x": value / r["fp64"]}
    if "fp64ph" in legs:
        r = lnl_rates(ev, BATCH, rank_seed(rank), args, flush, stream, (("f64ph", gwl.GWL_MIXED_F64PHASE),))
        legres["fp64ph_c2"] = {"v": r["f64ph"], "mixed_x": value / r["f64ph"]}
    if "grad" in legs:
        legres["grad_c5"] = leg_grad(ev, args, flush, stream, n_sm, fclk)
    if "cal" in legs:
        legres["cal_c2"] = leg_cal(ev, args, flush, stream, n_sm, fclk)
    if "calgrad" in legs:
        legres["calgrad_c2"] = leg_calgrad(ev, args, flush, stream)
    if "c1" in legs:
        legres["c1"] = lnl_rates(device_event("c1"), 1024, 1, args, flush, stream,
                                 (("mixed", gwl.GWL_MIXED), ("fp64", gwl.GWL_FP64)), local_fraction=0.0)
    if "c3" in legs:
        legres["c3"] = lnl_rates(device_event("c3"), 2048, 3, args, flush, stream,
                                 (("mixed", gwl.GWL_MIXED), ("fp64", gwl.GWL_FP64)))
    if "ns" in legs:
        legres["ns_c1"] = leg_ns()
        legres["eq5"] = leg_eq5()
    if "c5" in legs:
        legres["c5_ess"] = leg_c5(ev, args)
    if "c4" in legs:
        legres["c4"] = leg_c4(args, flush, stream)
    checks = out["cpu_baseline"].pop("checks") if "cpu_baseline" in out else None
    if legres or checks:
        # last in the line and compact, so that a reader keeping only the line's tail still has them
        out["legs"] = compact_legs(legres, checks)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def compact_legs(legres, checks):
    """The extra measurements in a short form (four significant digits):
      fp64_c2, fp64ph_c2  [evals/s, times slower than the mixed path]
      grad_c5, cal_c2     [evals/s, bin-loop ms, roofline fraction of the bound pipe]
      calgrad_c2          [grad evals/s, ms per call, gradient bin-loop ms, calibration-moment ms]
      c1, c3              [mixed evals/s, FP64 evals/s]
      ns_c1               [wall s, lnZ, its error, consumed per round / K ln(1 + B/K)]
      eq5                 [[B, consumed / K ln(1 + B/K), wall s], ...]
      c5                  {dims: {walk: [ESS/s, lnZ, lnZ spread over seeds]}}
      c4                  [batched / per-event lnL speed-up, NS s in one graph, NS s per event, rounds,
                           largest lnZ difference between the two in sigma]
      err_c1..c3          [FP64 |dlnL|, mixed |dlnL|, FP64-phase mixed |dlnL|, rows] against the oracle
      ns_c1_orc           [the oracle's NS wall s, lnZ]
      c4_lnZ              [[duration s, device lnZ, oracle lnZ, sigma], ...]"""
    L = {}
    g = legres.get
    if g("fp64_c2"):
        L["fp64_c2"] = [g("fp64_c2")["v"], g("fp64_c2")["mixed_x"]]
    if g("fp64ph_c2"):
        L["fp64ph_c2"] = [g("fp64ph_c2")["v"], g("fp64ph_c2")["mixed_x"]]
    if g("grad_c5"):
        L["grad_c5"] = [g("grad_c5")["v"], g("grad_c5")["kernel_ms"], g("grad_c5")["frac"]]
    if g("cal_c2"):
        L["cal_c2"] = [g("cal_c2")["v"], g("cal_c2")["kernel_ms"], g("cal_c2")["frac"]]
    if g("calgrad_c2"):
        c = g("calgrad_c2")
        L["calgrad_c2"] = [c["v"], c["ms"], c["grad_bins_ms"], c["cal_moments_ms"]]
    for k in ("c1", "c3"):
        if g(k):
            L[k] = [g(k)["mixed"], g(k)["fp64"]]
    if g("ns_c1"):
        n = g("ns_c1")
        L["ns_c1"] = [n["wall_s"], n["lnZ"], n["lnZ_err"], n["consumed"] / n["eq5"]]
    if g("eq5"):
        L["eq5"] = [[r[0], r[1], r[3]] for r in g("eq5")["rows"]]
    if g("c5_ess"):
        L["c5"] = {d: {w: [v["ess_s"], v["lnZ"], v["spread"]] for w, v in row.items()} for d, row in g("c5_ess").items()}
    if g("c4"):
        c = g("c4")
        L["c4"] = [c["lnl_x"], c["ns_graph_s"], c["ns_per_event_s"], c["rounds"], c["lnZ_graph_vs_per_event_max_sigma"]]
    if checks:
        for k in ("c1", "c2", "c3"):
            if k in checks:
                L["err_" + k] = [checks[k]["fp64"], checks[k]["mixed"], checks[k]["f64ph"], checks[k]["rows"]]
        if "ns_c1_oracle" in checks:
            o = checks["ns_c1_oracle"]
            L["ns_c1_orc"] = [o["wall_s"], o["lnZ"]]
        if "c4_lnZ" in checks:
            L["c4_lnZ"] = [[r["T"], r["dev"], r["orc"], r["sigma"]] for r in checks["c4_lnZ"]]
    return r4(L)


# ---------------------------------------------------------------- oracle (host cores): baseline and checks
def oracle_event(name=CONFIG, seed=SEED, cfg=None):
    import oracle

    def wf(ev, th):
        return oracle.waveform(ev, th)

    def snr2(ev, th):
        return -2.0 * oracle.loglike(ev.with_strain(np.zeros_like(ev.strain)), th[None])[0]

    return I.make_event(name, seed, wf, snr2, cfg=cfg)


def max_err(ev, theta_full, ref):
    """max |lnL_device - lnL_oracle| of both device paths on the oracle's own event (bars 1e-6 / 1e-3)."""
    import torch

    from paper_1909_11873_gb300 import gwl

    x = torch.from_numpy(np.ascontiguousarray(I.reduced(theta_full, ev.sampling))).cuda()
    out = {"rows": int(theta_full.shape[0])}
    for name, prec in (("fp64", gwl.GWL_FP64), ("mixed", gwl.GWL_MIXED), ("f64ph", gwl.GWL_MIXED_F64PHASE)):
        ctx = gwl.Context.from_event(ev, prec)
        got = gwl.loglike(ctx, x).cpu().numpy()
        ctx.gwl_sync()
        ctx.close()
        out[name] = float(np.max(np.abs(got - ref)))
        out[name + "_rel"] = float(np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))))
    return out


def cpu_baseline(theta_full, seconds, legs):
    """The FP64 oracle (as it stands) on all host cores, repeated over the batch until ~seconds elapse; then
    the oracle comparisons of the device legs (|dlnL| per workload, nested-sampling evidence)."""
    import oracle

    ev = oracle_event()
    n = os.cpu_count() or 1
    sample = theta_full[:1024]
    t0 = time.perf_counter()
    done = 0
    while True:
        ref = oracle.loglike(ev, sample, n_threads=n)
        done += sample.shape[0]
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    checks = {"bars": [1e-6, 1e-3], "c2": max_err(ev, sample, ref)}
    if "c1" in legs:
        e1 = oracle_event("c1", 1)
        th = I.proposals(e1, 1024, 1, local_fraction=0.0)
        checks["c1"] = max_err(e1, th, oracle.loglike(e1, th, n_threads=n))
    if "c3" in legs:
        e3 = oracle_event("c3", 3)
        th = I.proposals(e3, 2048, 3)[::32]  # 64 of the 2048 rows
        checks["c3"] = max_err(e3, th, oracle.loglike(e3, th, n_threads=n))
    if "ns" in legs:
        e1 = oracle_event("c1", SEED)
        t1 = time.perf_counter()
        r = oracle.ns_run(e1, e1.sampling, NS_K, NS_CHAINS, NS_WALK, seed=2, dlogz=0.1)
        checks["ns_c1_oracle"] = {"wall_s": time.perf_counter() - t1, "lnZ": r["lnZ"], "lnZ_err": r["lnZ_err"]}
    if "c4" in legs:
        checks["c4_lnZ"] = c4_oracle_lnz(n)
    return {"value": done / el, "unit": "evals/s", "cores": n, "kind": "oracle",
            "sample": f"{done} evaluations = repeated first 1024 proposals of the 8192-proposal batch "
                      f"(same event, oracle-made injection), {el:.1f} s wall", "checks": checks}


def c4_oracle_lnz(n_threads):
    """lnZ of the device's full-scale run (K = 1000, 1000 chains, walk 100, 4-D) against the oracle's on the
    two shortest BBH events of the 64-event workload (oracle-made injections, same data for both)."""
    from paper_1909_11873_gb300 import gwl
    import oracle

    cfgs = I.c4_events(C4_SEED, 64)
    pick = sorted((c["T"], i) for i, c in enumerate(cfgs) if c["source"] == "bbh")[:2]
    rows = []
    for _, i in pick:
        c = cfgs[i]
        ev = four_d(oracle_event("custom", c["seed"], cfg=c))
        ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
        d = ctx.ns_run(C4_K, C4_CHAINS, C4_WALK, seed=C4_SEED + 1 + i, dlogz=0.1)
        ctx.close()
        t0 = time.perf_counter()
        o = oracle.ns_run(ev, ev.sampling, C4_K, C4_CHAINS, C4_WALK, seed=C4_SEED + 101 + i, dlogz=0.1)
        rows.append({"event": i, "T": c["T"], "dev": d["lnZ"], "orc": o["lnZ"],
                     "sigma": math.hypot(d["lnZ_err"], o["lnZ_err"]), "oracle_s": time.perf_counter() - t0})
    return rows


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


def run_profile_only(args):
    """One workload's calls, untimed, for a profiler; the launch shape from --shape (else the defaults)."""
    import torch

    from paper_1909_11873_gb300 import build, gwl

    if not os.path.exists(gwl.LIB_PATH):
        build.build()
    torch.cuda.set_device(0)
    if args.profile_only == "ns":
        return run_profile_ns(args)
    ev = device_event(args.profile_config)
    prec = {"fp64ph": gwl.GWL_MIXED_F64PHASE, "fp64": gwl.GWL_FP64}.get(args.profile_only, gwl.GWL_MIXED)
    ctx = gwl.Context.from_event(ev, prec)
    grad = args.profile_only in ("grad", "calgrad")
    B = 4096 if grad else (2048 if args.profile_config == "c3" else BATCH)
    if args.profile_only in ("cal", "calgrad"):
        th = I.calibrated_proposals(ev, B, SEED + (13 if grad else 11))
        rows = np.concatenate([I.reduced(th[:, :11], ev.sampling), th[:, 11:]], axis=1)
        ctx.gwl_set_calibration(I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1])))
    else:
        rows = I.reduced(I.proposals(ev, B, SEED + (7 if grad else 0)), ev.sampling)
    if args.shape:
        w, c = (int(v) for v in args.shape.split(","))
        ctx.gwl_set_tuning(window=0 if grad else w, ctas_per_sm=c, grad_window=w if grad else 0,
                           bin_kernel=args.bin_kernel)
    x = torch.from_numpy(np.ascontiguousarray(rows)).cuda()
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    for _ in range(args.warmup + args.steps):
        if grad:
            ctx.gwl_grad(x, out, g)
        else:
            ctx.gwl_loglike(x, out)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    print(json.dumps({"profile_only": args.profile_only, "calls": args.warmup + args.steps, "B": B,
                      "tuning": ctx.gwl_get_tuning(), "lnl0": float(out[0])}))
    ctx.close()


def run_profile_ns(args):
    """Device nested sampling on the 1-detector 4 s event (K = 250, 250 chains, walk 20): a warm-up run
    of --warmup rounds, then one of --steps rounds, timed by the host clock (per round and per walk
    step) -- the launch sequence of the sampler's rounds for a profiler's launch list."""
    from paper_1909_11873_gb300 import gwl

    ctx = gwl.Context.from_event(device_event("c1"), gwl.GWL_MIXED)
    ctx.ns_run(NS_K, NS_CHAINS, NS_WALK, seed=1, dlogz=0.0, max_rounds=max(args.warmup, 1))
    t0 = time.perf_counter()
    r = ctx.ns_run(NS_K, NS_CHAINS, NS_WALK, seed=2, dlogz=0.0, max_rounds=args.steps)
    wall = time.perf_counter() - t0
    n = int(r["rounds"])
    print(json.dumps({"profile_only": "ns", "rounds": n, "wall_ms": wall * 1e3,
                      "ms_per_round": wall * 1e3 / max(n, 1), "us_per_step": wall * 1e6 / max(n * NS_WALK, 1),
                      "launches": ctx.launch_count()}))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_only:
        run_profile_only(args)
    else:
        run_gwl(args)


if __name__ == "__main__":
    main()
