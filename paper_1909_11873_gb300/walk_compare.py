"""Random walk vs gradient-informed (Galilean) walk inside nested sampling.

  python -m paper_1909_11873_gb300.walk_compare [--config c5] [--dims 4|11] [--K 500] [--walk 20] [--seeds 3]

For each walk kind: wall time, lnZ and its error, the spread of lnZ over seeds,
and the Kish effective sample size of the posterior weights, ESS = (sum w)^2 /
sum w^2, over dead points and the final live set; effective samples per
second = ESS / wall time.  --dims 4 samples (Mc, q, tc, phic) with the other
parameters at the injection.  Events are seeded and made with the library's
own template.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c5")
    ap.add_argument("--dims", type=int, default=4, choices=[4, 11])
    ap.add_argument("--K", type=int, default=500)
    ap.add_argument("--walk", type=int, default=20)
    ap.add_argument("--seeds", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    a = ap.parse_args()
    from . import build, gwl
    from . import inputs as I
    from .profile_run import device_event

    build.build()
    ev = device_event(a.config, 2)
    if a.dims == 4:
        th = ev.theta_inj
        smp = I.Sampling(np.array([0, 1, 9, 10], dtype=np.int32), th.copy(), np.zeros(4, dtype=np.int32),
                         np.array([th[0] * 0.97, 0.25, -0.02, 0.0]), np.array([th[0] * 1.03, 1.0, 0.02, 2 * math.pi]),
                         np.array([0, 0, 0, 1], dtype=np.int32))
        ev = dataclasses.replace(ev, sampling=smp)
    prec = gwl.GWL_MIXED if a.precision == "mixed" else gwl.GWL_FP64
    out = {"config": a.config, "dims": a.dims, "K": a.K, "walk": a.walk, "precision": a.precision}
    for name, kind in (("random", gwl.GWL_WALK_RANDOM), ("galilean", gwl.GWL_WALK_GALILEAN)):
        ctx = gwl.Context.from_event(ev, prec)
        ctx.gwl_set_walk(kind)
        ctx.ns_run(a.K, a.K, a.walk, seed=999, dlogz=0.1, max_rounds=1)  # warm-up
        runs = []
        for sd in range(a.seeds):
            t0 = time.perf_counter()
            r = ctx.ns_run(a.K, a.K, a.walk, seed=100 + sd, dlogz=0.1, max_dead=400000)
            wall = time.perf_counter() - t0
            lw = r["dead_lnl"] + r["dead_logwt"]
            w = np.exp(lw - lw.max())
            ess = w.sum() ** 2 / (w ** 2).sum()
            runs.append(dict(wall_s=wall, lnZ=r["lnZ"], lnZ_err=r["lnZ_err"], ess=ess, rounds=r["rounds"],
                             acceptance=r["acceptance"], ess_per_s=ess / wall))
        lnz = np.array([x["lnZ"] for x in runs])
        out[name] = {"runs": runs, "lnZ_mean": float(lnz.mean()), "lnZ_spread": float(lnz.std(ddof=1)) if len(runs) > 1 else None,
                     "ess_per_s_mean": float(np.mean([x["ess_per_s"] for x in runs])),
                     "wall_s_mean": float(np.mean([x["wall_s"] for x in runs]))}
        ctx.close()
    out["galilean_over_random_ess_per_s"] = out["galilean"]["ess_per_s_mean"] / out["random"]["ess_per_s_mean"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
