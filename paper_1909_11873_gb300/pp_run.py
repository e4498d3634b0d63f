"""Probability-probability (PP) coverage test of the device nested sampler.

  python -m paper_1909_11873_gb300.pp_run [--n 100] [--K 250] [--walk 20] [--precision mixed]

N injections are drawn from a fixed 4-D prior (chirp mass, mass ratio, coalescence
time, phase) on the three-detector 8 s BBH network with coloured noise
(inputs.make_pp_event); for each, ns_run samples the same prior and the
credible level of the true value, C_k = sum_i w_i [theta_i,k < theta_true,k] /
sum_i w_i over the weighted dead points (and the final live set), is recorded.
If the sampler's posteriors are calibrated, each parameter's C_k is uniform on
[0, 1]: this script reports the Kolmogorov-Smirnov statistic and p-value per
parameter and Fisher's combination.  Injections are made with the library's
own template.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

NAMES = ("mc", "q", "tc", "phic")


def ks_uniform(x: np.ndarray) -> tuple[float, float]:
    """One-sample Kolmogorov-Smirnov statistic against U(0, 1) and its asymptotic p-value."""
    x = np.sort(np.asarray(x, dtype=np.float64))
    n = x.size
    i = np.arange(1, n + 1)
    d = float(max(np.max(i / n - x), np.max(x - (i - 1) / n)))
    lam = (math.sqrt(n) + 0.12 + 0.11 / math.sqrt(n)) * d  # Stephens' finite-n correction
    p = 2.0 * sum((-1) ** (k - 1) * math.exp(-2.0 * k * k * lam * lam) for k in range(1, 101))
    return d, float(min(max(p, 0.0), 1.0))


def fisher(ps) -> float:
    """Fisher's combined p-value: -2 sum ln p ~ chi^2 with 2 len(ps) degrees of freedom."""
    x = -2.0 * sum(math.log(max(p, 1e-300)) for p in ps)
    k = len(ps)  # chi^2 survival with 2k dof: e^{-x/2} sum_{j<k} (x/2)^j / j!
    h = x / 2.0
    return float(math.exp(-h) * sum(h ** j / math.factorial(j) for j in range(k)))


def credible_levels(n: int, K: int, walk: int, precision: str, seed0: int = 0, log=None) -> np.ndarray:
    """[n, 4] credible levels of the injected values, one device NS run per injection."""
    import torch

    from . import build, gwl
    from . import inputs as I

    build.build()
    cache = {}

    def waveform(ev, th):
        if "z" not in cache:  # zero-strain FP64 context over the full 11-D vector, shared by all events
            full = I.Sampling(np.arange(11, dtype=np.int32), np.zeros(11), np.zeros(11, dtype=np.int32),
                              np.zeros(11), np.ones(11), np.zeros(11, dtype=np.int32))
            cache["z"] = gwl.Context(ev.freqs, np.zeros_like(ev.strain), ev.psd, ev.geom, gwl.GWL_FP64,
                                     ev.fcut_mode, ev.gmst, ev.t_ref, full)
        h = gwl.waveform(cache["z"], torch.from_numpy(np.ascontiguousarray(th[None])).cuda()).cpu().numpy()[0]
        return h[..., 0] + 1j * h[..., 1]

    prec = gwl.GWL_MIXED if precision == "mixed" else gwl.GWL_FP64
    out = np.zeros((n, 4))
    for i in range(n):
        ev = I.make_pp_event(seed0 + i, waveform)
        smp = ev.sampling
        ctx = gwl.Context.from_event(ev, prec)
        r = ctx.ns_run(K, K, walk, seed=7_000 + seed0 + i, dlogz=0.1, max_dead=200_000)
        ctx.close()
        th = smp.lo + r["dead_u"] * (smp.hi - smp.lo)  # uniform priors on all four
        lw = r["dead_logwt"]
        w = np.exp(lw - lw.max())
        truth = ev.theta_inj[smp.param_map]
        out[i] = (w[:, None] * (th < truth[None, :])).sum(0) / w.sum()
        if log:
            log(f"{i:3d} lnZ {r['lnZ']:.2f} +- {r['lnZ_err']:.2f} dead {r['n_dead_returned']} "
                f"C = {np.array2string(out[i], precision=3)}")
    for c in cache.values():
        c.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=100)
    ap.add_argument("--K", type=int, default=250)
    ap.add_argument("--walk", type=int, default=20)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--seed0", type=int, default=0)
    a = ap.parse_args()
    C = credible_levels(a.n, a.K, a.walk, a.precision, a.seed0, log=lambda s: print(s, flush=True))
    res = {}
    for k, name in enumerate(NAMES):
        d, p = ks_uniform(C[:, k])
        res[name] = {"ks": d, "p": p}
    summary = dict(n=a.n, K=a.K, walk=a.walk, precision=a.precision, per_param=res,
                   fisher_p=fisher([v["p"] for v in res.values()]), levels=C.tolist())
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
