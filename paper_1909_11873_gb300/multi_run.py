"""Measure the many-events workload: 64 events of {4..128} s, 3 detectors, 20-1024 Hz, BBH or BNS.

  python -m paper_1909_11873_gb300.multi_run [--events 64] [--per 1000] [--walk 100] [--ns-rounds 2]

Reports (1) one batched multi-event lnL call over `per` proposals of every event
against the same proposals evaluated event by event (64 launch sequences), and
(2) the time of nested-sampling rounds (K = per, `per` chains, `walk` steps)
run for all events in one captured graph.  Events and injections are seeded
and made with the library's own template.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=64)
    ap.add_argument("--per", type=int, default=1000)
    ap.add_argument("--walk", type=int, default=100)
    ap.add_argument("--ns-rounds", type=int, default=2)
    ap.add_argument("--seed", type=int, default=4)
    a = ap.parse_args()
    import torch

    from . import build, gwl
    from . import inputs as I
    from .profile_run import device_event

    build.build()
    cfgs = I.c4_events(a.seed, a.events)
    evs, ths, ctxs = [], [], []
    t0 = time.perf_counter()
    for i, cfg in enumerate(cfgs):
        I.CONFIGS[f"_c4_{i}"] = cfg
        ev = device_event(f"_c4_{i}", cfg["seed"])
        evs.append(ev)
        ths.append(I.proposals(ev, a.per, cfg["seed"]))
        ctxs.append(gwl.Context.from_event(ev, gwl.GWL_MIXED))
    t_build = time.perf_counter() - t0
    mc = gwl.MultiContext(ctxs)
    x = torch.from_numpy(np.concatenate([I.reduced(t, ev.sampling) for t, ev in zip(ths, evs)])).cuda()
    xs = [x[i * a.per:(i + 1) * a.per] for i in range(a.events)]
    out = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
    fisco = []
    for ev, th in zip(evs, ths):
        eta = th[:, 1] / (1 + th[:, 1]) ** 2
        fi = 1 / (6 ** 1.5 * np.pi * th[:, 0] * eta ** -0.6 * 4.925490947e-6)
        fisco.append(np.searchsorted(ev.freqs, fi, side="right").sum() * ev.n_det)
    pairs = float(np.sum(fisco))

    def timeit(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_multi = timeit(lambda: mc.gwl_multi_loglike(x, out))
    ref = out.clone()
    outs = [torch.empty(a.per, dtype=torch.float64, device="cuda") for _ in range(a.events)]
    ms_each = timeit(lambda: [c.gwl_loglike(xx, o) for c, xx, o in zip(ctxs, xs, outs)])
    same = float((torch.cat(outs) - ref).abs().max())
    t0 = time.perf_counter()
    res = mc.gwl_multi_ns_run(a.per, a.per, a.walk, seed=a.seed, dlogz=0.1, max_rounds=a.ns_rounds)
    t_ns = time.perf_counter() - t0
    durations = [c["T"] for c in cfgs]
    print(json.dumps({
        "events": a.events, "per_event": a.per, "durations_s": durations,
        "sources": [c["source"] for c in cfgs], "event_build_s": t_build,
        "batched_ms": ms_multi, "per_event_launches_ms": ms_each, "batched_speedup": ms_each / ms_multi,
        "batched_evals_per_s": a.events * a.per / (ms_multi * 1e-3),
        "detector_bin_evals_per_s": pairs / (ms_multi * 1e-3), "max_abs_diff_vs_per_event": same,
        "ns_rounds": int(max(r["rounds"] for r in res)), "ns_wall_s": t_ns,
        "ns_s_per_round": t_ns / max(1, max(r["rounds"] for r in res)),
        "ns_walk": a.walk, "ns_K": a.per,
    }))


if __name__ == "__main__":
    main()
