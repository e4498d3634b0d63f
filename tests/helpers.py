"""Shared test helpers: events built with the oracle's own waveform (tests may use the oracle)."""
import functools

import numpy as np

import oracle
from paper_1909_11873_gb300 import inputs as I


def oracle_waveform(ev, th):
    return oracle.waveform(ev, th)


def oracle_snr2(ev, th):
    return -2.0 * oracle.loglike(ev.with_strain(np.zeros_like(ev.strain)), th[None])[0]


@functools.lru_cache(maxsize=None)
def event(name, seed=1, fcut_mode=0):
    return I.make_event(name, seed, oracle_waveform, oracle_snr2, fcut_mode=fcut_mode)


def custom_event(cfg, seed, fcut_mode=0):
    return I.make_event("custom", seed, oracle_waveform, oracle_snr2, cfg=cfg, fcut_mode=fcut_mode)


def tol(precision, ref):
    """|dlnL| bound, absolute at every |lnL|: 1e-6 for the FP64 path, 1e-3 for the mixed paths."""
    base = 1e-6 if precision == 0 else 1e-3
    return np.full(np.shape(ref), base)
