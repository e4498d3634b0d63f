"""Per-configuration |dlnL| of the device paths against the FP64 oracle (a report, not a test).

  python tests/report_precision.py

Prints, for each workload, the number of rows compared and the largest and
median absolute difference of GWL_FP64 and GWL_MIXED, plus the mixed path's
largest difference relative to |lnL|.  Rows are sampled from the full batch
evaluated on the device.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from helpers import event  # noqa: E402
from paper_1909_11873_gb300 import build, gwl  # noqa: E402
from paper_1909_11873_gb300 import inputs as I  # noqa: E402


def main():
    import torch

    build.build()
    rows = {"c1": (1024, 1024), "c2": (8192, 1024), "c3": (2048, 48)}
    for name, (B, n) in rows.items():
        ev = event(name)
        th = I.proposals(ev, B, 3, local_fraction=0.0 if name == "c1" else 0.5)
        idx = np.random.default_rng(0).choice(B, n, replace=False)
        ref = oracle.loglike(ev, th[idx])
        line = [f"{name}: B={B}, rows compared {n}, |lnL| up to {np.abs(ref).max():.3g}"]
        for prec in (0, 1):
            ctx = gwl.Context.from_event(ev, prec)
            got = gwl.loglike(ctx, torch.from_numpy(I.reduced(th, ev.sampling)).cuda()).cpu().numpy()[idx]
            ctx.gwl_sync()
            d = np.abs(got - ref)
            line.append(f"{'fp64' if prec == 0 else 'mixed'} max {d.max():.2e} median {np.median(d):.2e} "
                        f"max rel {np.max(d / np.maximum(np.abs(ref), 1.0)):.2e}")
        print("; ".join(line), flush=True)
    # the calibration model (ten nodes per detector over the band)
    for name, (B, n) in {"c1": (1024, 1024), "c2": (8192, 1024), "c3": (2048, 24)}.items():
        ev = event(name)
        th = I.calibrated_proposals(ev, B, 4)
        nodes = I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1]))
        idx = np.random.default_rng(1).choice(B, n, replace=False)
        ref = oracle.loglike_cal(ev, nodes, th[idx])
        rows_dev = np.ascontiguousarray(np.concatenate([I.reduced(th[:, :11], ev.sampling), th[:, 11:]], axis=1))
        line = [f"{name} calibrated ({rows_dev.shape[1]} parameters per row): B={B}, rows compared {n}"]
        for prec in (0, 1):
            ctx = gwl.Context.from_event(ev, prec)
            ctx.gwl_set_calibration(nodes)
            got = gwl.loglike(ctx, torch.from_numpy(rows_dev).cuda()).cpu().numpy()[idx]
            ctx.gwl_sync()
            d = np.abs(got - ref)
            line.append(f"{'fp64' if prec == 0 else 'mixed'} max {d.max():.2e} median {np.median(d):.2e}")
        print("; ".join(line), flush=True)


if __name__ == "__main__":
    main()
