"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access (ctypes) to ``gwl_oracle.cpp``: the plain per-bin definition of
the frequency-domain Gaussian-noise log-likelihood (Eq. 2 of Smith et al.
2020, read as the log-likelihood ratio), the same with the per-detector
calibration model of Section 2.2, its dual-number gradient, a plain
static parallel nested sampler (Section 3, Algorithm 1) with its constrained
random walk, and the gradient-informed (Galilean) constrained walk.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.

Parity status: the non-spinning phase through 3.5PN is pinned by its published
coefficients; the spin-orbit phase terms (1.5, 2.5, 3 and 3.5PN) by a
stationary-phase derivation from the published spin-orbit binding energy and
flux; everything else by closed forms, invariants, brute force or library
routines in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "gwl_oracle.cpp")
_lock = threading.Lock()
_lib = None

N_PARAM = 11
PARAM_NAMES = ("mc", "q", "chi1", "chi2", "dl", "iota", "psi", "ra", "dec", "tc", "phic")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O3, OpenMP, no -ffast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O3", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            d, i64, i32, u64 = C.c_double, C.c_int64, C.c_int, C.c_uint64
            P = C.c_void_p
            _lib.oracle_waveform.argtypes = [P, i64, P, i32, d, d, i32, P, P]
            _lib.oracle_antenna.argtypes = [P, i32, d, d, d, d, P]
            _lib.oracle_pn_psi.argtypes = [d, d, d, d, d]
            _lib.oracle_pn_psi.restype = d
            _lib.oracle_loglike.argtypes = [P, i64, P, P, P, i32, d, d, i32, P, i64, P, i32]
            _lib.oracle_grad.argtypes = [P, i64, P, P, P, i32, d, d, i32, P, i64, P, P, i32]
            _lib.oracle_loglike_cal.argtypes = [P, i64, P, P, P, i32, d, d, i32, i32, P, P, i64, P, i32]
            _lib.oracle_cal_spline.argtypes = [i32, P, P, i64, P, P]
            _lib.oracle_grad_cal.argtypes = [P, i64, P, P, P, i32, d, d, i32, i32, P, P, i64, P, P, i32]
            _lib.oracle_inv_normal_cdf.argtypes = [i64, P, P]
            _lib.oracle_ns_replace_cal.argtypes = ([P, i64, P, P, P, i32, d, d, i32, i32, P, P, P, P, P, P]
                                                   + [i32, P, P]
                                                   + [P, P, i64, i64, d, u64, u64, i64, i32, d, P, P, P, P, P, i32])
            _lib.oracle_ns_run_cal.argtypes = ([P, i64, P, P, P, i32, d, d, i32, i32, P, P, P, P, P, P]
                                               + [i32, P, P, i64, i64, i32, u64, d, i64, d, P, i32])
            _lib.oracle_philox.argtypes = [P, P, P]
            _lib.oracle_prior_transform.argtypes = [i32, P, P, P, P, P, P, P, i64, P]
            _lib.oracle_ns_replace.argtypes = ([P, i64, P, P, P, i32, d, d, i32, i32, P, P, P, P, P, P]
                                               + [P, P, i64, i64, d, u64, u64, i64, i32, d, P, P, P, P, P, i32])
            _lib.oracle_ns_run.argtypes = ([P, i64, P, P, P, i32, d, d, i32, i32, P, P, P, P, P, P]
                                           + [i64, i64, i32, u64, d, i64, d, P, P, P, P, i64, i32])
            _lib.oracle_ns_run_gauss.argtypes = [i32, P, d, i64, i64, i32, u64, d, i64, d, P, P, P, P, i64, i32]
            _lib.oracle_gmc_replace.argtypes = ([P, i64, P, P, P, i32, d, d, i32, i32, P, P, P, P, P, P]
                                                + [i32, P, P]
                                                + [P, P, i64, i64, d, u64, u64, i64, i32, d, d, P, P, P, P, P, i32])
            _lib.oracle_unit_grad.argtypes = ([P, i64, P, P, P, i32, d, d, i32, i32, P, P, P, P, P, P]
                                              + [i32, P, P, P, i64, P, P, i32])
            _lib.oracle_gmc_gauss.argtypes = [i32, P, d, P, P, i64, d, u64, u64, i32, d, d, P, P, P, P, i32]
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _ev_args(ev):
    """(freqs, M, strain[n_det][M][2], psd, geom, n_det, gmst, t_ref, fcut_mode)."""
    freqs = _f64(ev.freqs)
    strain = np.ascontiguousarray(np.stack([ev.strain.real, ev.strain.imag], axis=-1), dtype=np.float64)
    psd = _f64(ev.psd)
    geom = _f64(ev.geom)
    keep = (freqs, strain, psd, geom)
    return keep, [_p(freqs), freqs.size, _p(strain), _p(psd), _p(geom), geom.shape[0], ev.gmst, ev.t_ref,
                  ev.fcut_mode]


def _smp_args(smp):
    pm = _i32(smp.param_map)
    fx = _f64(smp.fixed)
    kd = _i32(smp.kind)
    lo = _f64(smp.lo)
    hi = _f64(smp.hi)
    pe = _i32(smp.periodic)
    keep = (pm, fx, kd, lo, hi, pe)
    return keep, [len(pm), _p(pm), _p(fx), _p(kd), _p(lo), _p(hi), _p(pe)]


def waveform(ev, theta) -> np.ndarray:
    """Per-bin detector strain h_d(f_j) -> complex128 [n_det, M] (11-D theta)."""
    th = _f64(theta).reshape(N_PARAM)
    freqs = _f64(ev.freqs)
    geom = _f64(ev.geom)
    h = np.zeros((geom.shape[0], freqs.size, 2))
    _L().oracle_waveform(_p(freqs), freqs.size, _p(geom), geom.shape[0], ev.gmst, ev.t_ref, ev.fcut_mode,
                         _p(th), _p(h))
    return h[..., 0] + 1j * h[..., 1]


def antenna(geom, gmst, psi, ra, dec) -> np.ndarray:
    """[n_det, 3] = (F+, Fx, arrival delay dt [s]) per detector."""
    g = _f64(geom)
    out = np.zeros((g.shape[0], 3))
    _L().oracle_antenna(_p(g), g.shape[0], gmst, psi, ra, dec, _p(out))
    return out


def pn_psi(mc, q, chi1, chi2, f) -> float:
    return _L().oracle_pn_psi(mc, q, chi1, chi2, f)


def loglike(ev, theta, n_threads: int | None = None) -> np.ndarray:
    """lnL for theta[B, 11] -> [B] (FP64, per-bin definition)."""
    th = _f64(theta).reshape(-1, N_PARAM)
    out = np.zeros(th.shape[0])
    keep, a = _ev_args(ev)
    _L().oracle_loglike(*a, _p(th), th.shape[0], _p(out), n_threads or default_threads())
    return out


def grad(ev, theta, n_threads: int | None = None):
    """(lnL [B], d lnL / d theta [B, 11]) by forward-mode dual numbers."""
    th = _f64(theta).reshape(-1, N_PARAM)
    out = np.zeros(th.shape[0])
    g = np.zeros_like(th)
    keep, a = _ev_args(ev)
    _L().oracle_grad(*a, _p(th), th.shape[0], _p(out), _p(g), n_threads or default_threads())
    return out, g


def loglike_cal(ev, node_freqs, theta, n_threads: int | None = None) -> np.ndarray:
    """lnL with the calibration model for theta[B, 11 + 2 n_nodes n_det] -> [B].

    After the 11 source parameters each row holds, per detector, the amplitude
    corrections dA at the nodes and then the phase corrections dphi [rad]; the
    template of detector d is multiplied by (1 + dA_d(f)) exp(i dphi_d(f)),
    both natural cubic splines in ln f through the nodes (Section 2.2's
    calibration model, in the reading stated in gwl_oracle.cpp).
    """
    nf = _f64(node_freqs)
    n_det = np.asarray(ev.geom).shape[0]
    th = _f64(theta).reshape(-1, N_PARAM + 2 * nf.size * n_det)
    out = np.zeros(th.shape[0])
    keep, a = _ev_args(ev)
    rc = _L().oracle_loglike_cal(*a, nf.size, _p(nf), _p(th), th.shape[0], _p(out), n_threads or default_threads())
    if rc:
        raise ValueError("calibration needs at least two nodes")
    return out


def grad_cal(ev, node_freqs, theta, n_threads: int | None = None):
    """(lnL [B], d lnL / d theta [B, D]) with the calibration model, D = 11 + 2 n_nodes n_det:
    the derivatives with respect to the source parameters and to every node's amplitude and
    phase correction, by forward-mode dual numbers (the layout of loglike_cal)."""
    nf = _f64(node_freqs)
    n_det = np.asarray(ev.geom).shape[0]
    th = _f64(theta).reshape(-1, N_PARAM + 2 * nf.size * n_det)
    out = np.zeros(th.shape[0])
    g = np.zeros_like(th)
    keep, a = _ev_args(ev)
    rc = _L().oracle_grad_cal(*a, nf.size, _p(nf), _p(th), th.shape[0], _p(out), _p(g), n_threads or default_threads())
    if rc:
        raise ValueError("calibration needs at least two nodes")
    return out, g


def cal_spline(x, y, xq) -> np.ndarray:
    """The oracle's natural cubic spline through (x, y) evaluated at xq."""
    xx, yy, qq = _f64(x), _f64(y), _f64(xq)
    out = np.zeros(qq.size)
    _L().oracle_cal_spline(xx.size, _p(xx), _p(yy), qq.size, _p(qq), _p(out))
    return out


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _L().oracle_philox(_p(c), _p(k), _p(o))
    return o


def prior_transform(smp, u) -> np.ndarray:
    """Unit cube u[n, D] -> theta[n, 11]."""
    uu = _f64(u).reshape(-1, len(smp.param_map))
    out = np.zeros((uu.shape[0], N_PARAM))
    keep, a = _smp_args(smp)
    _L().oracle_prior_transform(*a, _p(uu), uu.shape[0], _p(out))
    return out


def ns_replace(ev, smp, live_u, live_lnl, worst, lnl_star, seed, counter, n_chains, walk_len, scale, chol,
               n_threads: int | None = None):
    """Constrained random walks (same stream as the device sampler).

    Returns (out_u [n_chains, D], out_lnl [n_chains], out_nacc [n_chains], start [n_chains]).
    """
    D = len(smp.param_map)
    lu = _f64(live_u).reshape(-1, D)
    ll = _f64(live_lnl)
    ch = _f64(chol).reshape(D, D)
    ou = np.zeros((n_chains, D))
    ol = np.zeros(n_chains)
    on = np.zeros(n_chains, dtype=np.int32)
    os_ = np.zeros(n_chains, dtype=np.int32)
    k1, a = _ev_args(ev)
    k2, b = _smp_args(smp)
    rc = _L().oracle_ns_replace(*a, *b, _p(lu), _p(ll), lu.shape[0], int(worst), float(lnl_star), int(seed),
                                int(counter), int(n_chains), int(walk_len), float(scale), _p(ch), _p(ou), _p(ol),
                                _p(on), _p(os_), n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_ns_replace: bad arguments")
    return ou, ol, on, os_


NS_KEYS = ("lnZ", "lnZ_err", "H", "n_dead", "n_proposals", "rounds", "scale", "acceptance", "consumed_per_round")


def ns_run(ev, smp, K, n_chains, walk_len, seed, dlogz=0.1, max_rounds=100000, scale0=1.0, max_dead=0,
           n_threads: int | None = None):
    """Plain static parallel nested sampling on the GW likelihood."""
    res = np.zeros(9)
    D = len(smp.param_map)
    dl = np.zeros(max(max_dead, 1))
    dw = np.zeros(max(max_dead, 1))
    du = np.zeros((max(max_dead, 1), D))
    k1, a = _ev_args(ev)
    k2, b = _smp_args(smp)
    _L().oracle_ns_run(*a, *b, int(K), int(n_chains), int(walk_len), int(seed), float(dlogz), int(max_rounds),
                       float(scale0), _p(res), _p(dl), _p(dw), _p(du), int(max_dead),
                       n_threads or default_threads())
    out = dict(zip(NS_KEYS, res.tolist()))
    if max_dead:
        n = min(int(res[3]), max_dead)
        out.update(dead_lnl=dl[:n], dead_logwt=dw[:n], dead_u=du[:n])
    return out


def inv_normal_cdf(u) -> np.ndarray:
    """The oracle's standard normal quantile Phi^{-1}(u)."""
    uu = _f64(u).ravel()
    out = np.zeros(uu.size)
    _L().oracle_inv_normal_cdf(uu.size, _p(uu), _p(out))
    return out


def _cal_args(ev, cal):
    """cal = (node_freqs, sigma_amp, sigma_phase) -> (keep, args, calibration coordinates)."""
    nf = _f64(cal[0])
    sig = _f64([cal[1], cal[2]])
    n_det = np.asarray(ev.geom).shape[0]
    return (nf, sig), [nf.size, _p(nf), _p(sig)], 2 * nf.size * n_det


def ns_replace_cal(ev, smp, cal, live_u, live_lnl, worst, lnl_star, seed, counter, n_chains, walk_len, scale, chol,
                   n_threads: int | None = None):
    """ns_replace with the calibration model: walk coordinates are the sampled source coordinates followed by
    the calibration parameters (zero-mean Gaussian priors); cal = (node_freqs, sigma_amp, sigma_phase)."""
    k3, c, nc = _cal_args(ev, cal)
    D = len(smp.param_map) + nc
    lu = _f64(live_u).reshape(-1, D)
    ll = _f64(live_lnl)
    ch = _f64(chol).reshape(D, D)
    ou = np.zeros((n_chains, D))
    ol = np.zeros(n_chains)
    on = np.zeros(n_chains, dtype=np.int32)
    os_ = np.zeros(n_chains, dtype=np.int32)
    k1, a = _ev_args(ev)
    k2, b = _smp_args(smp)
    rc = _L().oracle_ns_replace_cal(*a, *b, *c, _p(lu), _p(ll), lu.shape[0], int(worst), float(lnl_star),
                                    int(seed), int(counter), int(n_chains), int(walk_len), float(scale), _p(ch),
                                    _p(ou), _p(ol), _p(on), _p(os_), n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_ns_replace_cal: bad arguments")
    return ou, ol, on, os_


def _walk_cal_args(ev, cal):
    """cal = None (no calibration model) or (node_freqs, sigma_amp, sigma_phase)."""
    if cal is None:
        return None, [0, None, None], 0
    return _cal_args(ev, cal)


GALILEAN_PERSISTENCE = 0.5


def gmc_replace(ev, smp, live_u, live_lnl, worst, lnl_star, seed, counter, n_chains, walk_len, scale, chol,
                cal=None, persistence=GALILEAN_PERSISTENCE, n_threads: int | None = None):
    """Galilean (gradient-informed) constrained walks on the device sampler's stream, optionally with the
    calibration model (cal as in ns_replace_cal); persistence = the velocity kept per step.  Returns
    (out_u, out_lnl, out_nacc, start) as ns_replace."""
    k3, c, nc = _walk_cal_args(ev, cal)
    D = len(smp.param_map) + nc
    lu = _f64(live_u).reshape(-1, D)
    ll = _f64(live_lnl)
    ch = _f64(chol).reshape(D, D)
    ou = np.zeros((n_chains, D))
    ol = np.zeros(n_chains)
    on = np.zeros(n_chains, dtype=np.int32)
    os_ = np.zeros(n_chains, dtype=np.int32)
    k1, a = _ev_args(ev)
    k2, b = _smp_args(smp)
    rc = _L().oracle_gmc_replace(*a, *b, *c, _p(lu), _p(ll), lu.shape[0], int(worst), float(lnl_star), int(seed),
                                 int(counter), int(n_chains), int(walk_len), float(scale), float(persistence), _p(ch),
                                 _p(ou), _p(ol), _p(on), _p(os_), n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_gmc_replace: bad arguments")
    return ou, ol, on, os_


def unit_grad(ev, smp, u, cal=None, n_threads: int | None = None):
    """lnL and d lnL / du at unit-cube points u [n, Dw] (Dw: sampled source coordinates, then the calibration
    coordinates when cal is given) -> (lnl [n], grad [n, Dw])."""
    k3, c, nc = _walk_cal_args(ev, cal)
    Dw = len(smp.param_map) + nc
    uu = _f64(u).reshape(-1, Dw)
    lnl = np.zeros(uu.shape[0])
    g = np.zeros_like(uu)
    k1, a = _ev_args(ev)
    k2, b = _smp_args(smp)
    if _L().oracle_unit_grad(*a, *b, *c, _p(uu), uu.shape[0], _p(lnl), _p(g), n_threads or default_threads()):
        raise ValueError("oracle_unit_grad: bad arguments")
    return lnl, g


def gmc_gauss(mu, sigma, periodic, u0, lnl_star, seed, counter, walk_len, scale, chol,
              persistence=GALILEAN_PERSISTENCE, n_threads: int | None = None):
    """Galilean walks on the Gaussian-in-a-box likelihood (ns_run_gauss's) from start points u0 [n, D]
    -> (out_u, out_lnl, out_nacc)."""
    m = _f64(mu)
    D = m.size
    pe = _i32(periodic)
    uu = _f64(u0).reshape(-1, D)
    ch = _f64(chol).reshape(D, D)
    ou = np.zeros_like(uu)
    ol = np.zeros(uu.shape[0])
    on = np.zeros(uu.shape[0], dtype=np.int32)
    if _L().oracle_gmc_gauss(D, _p(m), float(sigma), _p(pe), _p(uu), uu.shape[0], float(lnl_star), int(seed),
                             int(counter), int(walk_len), float(scale), float(persistence), _p(ch), _p(ou), _p(ol),
                             _p(on),
                             n_threads or default_threads()):
        raise ValueError("oracle_gmc_gauss: bad arguments")
    return ou, ol, on


def ns_run_cal(ev, smp, cal, K, n_chains, walk_len, seed, dlogz=0.1, max_rounds=100000, scale0=1.0,
               n_threads: int | None = None):
    """Plain static parallel nested sampling on the calibrated GW likelihood."""
    res = np.zeros(9)
    k3, c, nc = _cal_args(ev, cal)
    k1, a = _ev_args(ev)
    k2, b = _smp_args(smp)
    _L().oracle_ns_run_cal(*a, *b, *c, int(K), int(n_chains), int(walk_len), int(seed), float(dlogz),
                           int(max_rounds), float(scale0), _p(res), n_threads or default_threads())
    return dict(zip(NS_KEYS, res.tolist()))


def ns_run_gauss(D, mu, sigma, K, n_chains, walk_len, seed, dlogz=0.1, max_rounds=100000, scale0=1.0,
                 max_dead=0, n_threads: int | None = None):
    """Nested sampling of an isotropic Gaussian likelihood in the unit cube (with max_dead > 0, also
    the first max_dead dead points, final live points included: dead_lnl, dead_logwt, dead_u)."""
    res = np.zeros(9)
    m = _f64(mu)
    dl = np.zeros(max(max_dead, 1))
    dw = np.zeros(max(max_dead, 1))
    du = np.zeros((max(max_dead, 1), D))
    _L().oracle_ns_run_gauss(int(D), _p(m), float(sigma), int(K), int(n_chains), int(walk_len), int(seed),
                             float(dlogz), int(max_rounds), float(scale0), _p(res), _p(dl), _p(dw), _p(du),
                             int(max_dead), n_threads or default_threads())
    out = dict(zip(NS_KEYS, res.tolist()))
    if max_dead:
        n = min(int(res[3]), max_dead)
        out.update(dead_lnl=dl[:n], dead_logwt=dw[:n], dead_u=du[:n])
    return out
