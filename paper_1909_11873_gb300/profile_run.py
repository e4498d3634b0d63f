"""Run one workload through the library a fixed number of times (for profilers such as ncu).

  python -m paper_1909_11873_gb300.profile_run --config c2 --precision mixed --iters 5 [--entry loglike|grad]
      [--cal N]   (likelihood with the calibration model, N nodes per detector over the band)

The event is synthetic and seeded; its injection is produced by the library's
own template, so no test infrastructure is involved.
"""
from __future__ import annotations

import argparse

import numpy as np


def device_event(name, seed):
    import torch

    from . import gwl
    from . import inputs as I

    cache = {}

    def zctx(ev):
        if "c" not in cache:
            full = I.Sampling(np.arange(11, dtype=np.int32), np.zeros(11), np.zeros(11, dtype=np.int32),
                              np.zeros(11), np.ones(11), np.zeros(11, dtype=np.int32))
            cache["c"] = gwl.Context(ev.freqs, np.zeros_like(ev.strain), ev.psd, ev.geom, gwl.GWL_FP64, ev.fcut_mode,
                                     ev.gmst, ev.t_ref, full)
        return cache["c"]

    def waveform(ev, th):
        h = gwl.waveform(zctx(ev), torch.from_numpy(np.ascontiguousarray(th[None])).cuda()).cpu().numpy()[0]
        return h[..., 0] + 1j * h[..., 1]

    def snr2(ev, th):
        return -2.0 * float(gwl.loglike(zctx(ev), torch.from_numpy(np.ascontiguousarray(th[None])).cuda()).cpu()[0])

    ev = I.make_event(name, seed, waveform, snr2)
    for c in cache.values():
        c.close()
    return ev


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--entry", default="loglike", choices=["loglike", "grad"])
    ap.add_argument("--time", action="store_true", help="report device-timed evals/s (L2 flushed between calls)")
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--cal", type=int, default=0, help="calibration nodes per detector (0: off)")
    a = ap.parse_args()
    import torch

    from . import build, gwl
    from . import inputs as I

    build.build()
    ev = device_event(a.config, a.seed)
    B = a.batch or I.CONFIGS[a.config]["batch"]
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED if a.precision == "mixed" else gwl.GWL_FP64)
    if a.cal:
        full = I.calibrated_proposals(ev, B, a.seed, n_nodes=a.cal)
        rows = np.concatenate([I.reduced(full[:, :11], ev.sampling), full[:, 11:]], axis=1)
        ctx.gwl_set_calibration(I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1]), a.cal))
    else:
        rows = I.reduced(I.proposals(ev, B, a.seed), ev.sampling)
    th = torch.from_numpy(np.ascontiguousarray(rows)).cuda()
    ctx.gwl_set_tuning(window=a.window, ctas_per_sm=a.ctas)
    out = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(th)
    def call():
        if a.entry == "grad":
            ctx.gwl_grad(th, out, grad)
        else:
            ctx.gwl_loglike(th, out)

    for _ in range(a.iters):
        call()
    torch.cuda.synchronize()
    ctx.gwl_sync()
    msg = (f"{a.config} {a.precision} {a.entry} cal={a.cal} B={B} window={a.window} ctas={a.ctas} "
           f"iters={a.iters} lnL[0]={out[0].item():.6f}")
    if a.time:
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.iters)]
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record()
            call()
            e1.record()
        torch.cuda.synchronize()
        ms = sum(x.elapsed_time(y) for x, y in evs) / len(evs)
        msg += f" ms/call={ms:.4f} evals/s={B / (ms * 1e-3):.4e}"
    print(msg)


if __name__ == "__main__":
    main()
