"""Usable replacements per round and nested-sampling wall time against the batch size.

  python -m paper_1909_11873_gb300.eq5_run [--config c1] [--K 250] [--walk 20] [--batches 25,50,...] [--seeds 2]

With K live points and B candidates drawn per round above the round's first
threshold, the replacement loop consumes, on average, K ln(1 + B/K) of them
per round (Eq. 5): the speed-up of parallel sampling over one candidate per
round.  For each B this driver runs full device nested-sampling runs
(ns_run, random walk) on a seeded synthetic event and reports the measured
candidates consumed per round against K ln(1 + B/K), the rounds, the wall
time, lnZ and its error.  The event is made with the library's own template.
"""
from __future__ import annotations

import argparse
import json
import math
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c1")
    ap.add_argument("--K", type=int, default=250)
    ap.add_argument("--walk", type=int, default=20)
    ap.add_argument("--batches", default="25,50,125,250,500,1000,2000,4000")
    ap.add_argument("--seeds", type=int, default=2)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    a = ap.parse_args()
    from . import build, gwl
    from .profile_run import device_event

    build.build()
    ev = device_event(a.config, 2)
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED if a.precision == "mixed" else gwl.GWL_FP64)
    ctx.ns_run(a.K, 64, a.walk, seed=99, dlogz=0.1, max_rounds=2)  # warm-up (graphs, scratch)
    rows = []
    for B in (int(x) for x in a.batches.split(",")):
        runs = []
        for s in range(a.seeds):
            t0 = time.perf_counter()
            r = ctx.ns_run(a.K, B, a.walk, seed=1000 + s, dlogz=0.1)
            wall = time.perf_counter() - t0
            runs.append(dict(wall_s=wall, lnZ=r["lnZ"], lnZ_err=r["lnZ_err"], rounds=r["rounds"],
                             consumed_per_round=r["consumed_per_round"], n_dead=r["n_dead"],
                             proposals=r["n_proposals"]))
        eq5 = a.K * math.log(1.0 + B / a.K)
        mean = lambda k: sum(x[k] for x in runs) / len(runs)  # noqa: E731
        rows.append(dict(B=B, eq5=eq5, consumed_per_round=mean("consumed_per_round"),
                         ratio=mean("consumed_per_round") / eq5, rounds=mean("rounds"), wall_s=mean("wall_s"),
                         lnZ=mean("lnZ"), lnZ_err=mean("lnZ_err"), runs=runs))
        print(f"B={B:5d} Eq.5 {eq5:8.1f} measured {rows[-1]['consumed_per_round']:8.1f} "
              f"(x{rows[-1]['ratio']:.3f}) rounds {rows[-1]['rounds']:6.1f} wall {rows[-1]['wall_s'] * 1e3:8.1f} ms "
              f"lnZ {rows[-1]['lnZ']:.3f} +- {rows[-1]['lnZ_err']:.3f}", flush=True)
    ctx.close()
    print(json.dumps(dict(config=a.config, K=a.K, walk=a.walk, precision=a.precision, rows=rows)))


if __name__ == "__main__":
    main()
