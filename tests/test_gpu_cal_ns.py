"""Device random walks and nested sampling with the calibration model (Section 2.2) against the oracle.

With calibration, ns_replace and ns_run walk in the sampled source coordinates followed by the
2 n_nodes n_det calibration coordinates (zero-mean Gaussian priors, theta = sigma Phi^{-1}(u)).
"""
import math

import numpy as np
import pytest

import oracle
from helpers import event
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIG = (0.1, 0.1)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build
    build.build()


def nodes_for(ev, n):
    return I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1]), n)


def cal_theta(ev, nodes, u):
    """Full oracle rows [n, 11 + 2 n_nodes n_det] of unit-cube points [n, D + 2 n_nodes n_det]."""
    smp = ev.sampling
    th = oracle.prior_transform(smp, u[:, :smp.D])
    nn = nodes.size
    c = np.arange(u.shape[1] - smp.D)
    sig = np.where((c // nn) % 2 == 1, SIG[1], SIG[0])
    cal = sig[None, :] * oracle.inv_normal_cdf(u[:, smp.D:]).reshape(u.shape[0], -1)
    return np.concatenate([th, cal], axis=1)


def live_set(ev, nodes, K, seed):
    D = ev.sampling.D + 2 * nodes.size * ev.geom.shape[0]
    u = np.random.default_rng(seed).uniform(0, 1, (K, D))
    return u, oracle.loglike_cal(ev, nodes, cal_theta(ev, nodes, u))


def cal_ctx(ev, nodes, precision):
    from paper_1909_11873_gb300 import gwl
    ctx = gwl.Context.from_event(ev, precision)
    ctx.gwl_set_calibration(nodes, *SIG)
    return ctx


def device_walk(ctx, u, ll, worst, lstar, seed, counter, n, walk_len, scale, chol):
    D = u.shape[1]
    assert ctx.theta_stride == D
    ou = torch.zeros((n, D), dtype=torch.float64, device="cuda")
    ol = torch.zeros(n, dtype=torch.float64, device="cuda")
    on = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.ns_replace(torch.from_numpy(u).cuda(), torch.from_numpy(ll).cuda(), worst, lstar, seed, counter, n, walk_len,
                   scale, torch.from_numpy(np.ascontiguousarray(chol)).cuda(), ou, ol, on, os_)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    return ou.cpu().numpy(), ol.cpu().numpy(), on.cpu().numpy(), os_.cpu().numpy()


@pytest.mark.parametrize("cfg,n_nodes", [("c1", 4), ("c2", 10)])
def test_calibrated_ns_replace_replays_oracle_walk_fp64(cfg, n_nodes):
    """Same Philox stream, FP64 calibrated likelihood, 12-D (1 detector, 4 nodes) and 71-D (3 detectors,
    10 nodes) walks: identical start points and accept counts, end points to 1e-12."""
    ev = event(cfg)
    nodes = nodes_for(ev, n_nodes)
    K = 128
    u, ll = live_set(ev, nodes, K, 3)
    worst = int(np.argmin(ll))
    D = u.shape[1]
    chol = np.diag(np.full(D, 0.03))
    n, wl, seed, ctr = 160, 10, 0x51CA1B, 5
    ctx = cal_ctx(ev, nodes, 0)
    gu, gl, gn, gs = device_walk(ctx, u, ll, worst, ll[worst], seed, ctr, n, wl, 1.0, chol)
    ou, ol, on, os_ = oracle.ns_replace_cal(ev, ev.sampling, (nodes, *SIG), u, ll, worst, ll[worst], seed, ctr, n,
                                            wl, 1.0, chol)
    assert np.array_equal(gs, os_)
    assert np.array_equal(gn, on)
    assert np.allclose(gu, ou, rtol=0, atol=1e-12)
    assert np.allclose(gl, ol, rtol=0, atol=1e-6)
    assert gn.sum() > 0


def test_calibrated_ns_replace_mixed_properties():
    """Mixed precision, 71-D: every chain ends at its start or at a point whose oracle lnL is >= L* and
    equals the returned lnL within the mixed tolerance."""
    ev = event("c2")
    nodes = nodes_for(ev, 10)
    u, ll = live_set(ev, nodes, 128, 4)
    worst = int(np.argmin(ll))
    chol = np.diag(np.full(u.shape[1], 0.02))
    ctx = cal_ctx(ev, nodes, 1)
    gu, gl, gn, gs = device_walk(ctx, u, ll, worst, ll[worst], 99, 1, 192, 8, 1.0, chol)
    moved = gn > 0
    assert moved.any() and np.all(gs != worst)
    assert np.allclose(gu[~moved], u[gs[~moved]]) and np.allclose(gl[~moved], ll[gs[~moved]])
    ref = oracle.loglike_cal(ev, nodes, cal_theta(ev, nodes, gu[moved]))
    assert np.all(np.abs(ref - gl[moved]) <= 1e-3)
    assert np.all(ref >= ll[worst] - 1e-3)


def test_calibrated_ns_run_lnz_matches_oracle():
    """Device NS over 4 source + 8 calibration coordinates (K = 250, walk 60) vs the oracle's NS: the mean
    lnZ of two runs on each side.  (A constant calibration phase is degenerate with phi_c, a ridge that
    random-walk NS explores unevenly; at walk length 20 single runs scatter by more than sqrt(H/K).)"""
    ev = event("c1")
    nodes = nodes_for(ev, 4)
    K, nch, wl = 250, 250, 60
    ctx = cal_ctx(ev, nodes, 1)
    g = [ctx.ns_run(K, nch, wl, seed=s, dlogz=0.1, max_dead=20000) for s in (21, 23)]
    o = [oracle.ns_run_cal(ev, ev.sampling, (nodes, *SIG), K, nch, wl, seed=s, dlogz=0.1) for s in (22, 24)]
    for r in g:
        assert np.isfinite(r["lnZ"]) and r["rounds"] > 3
        assert r["dead_u"].shape[1] == 12
    gm = np.mean([r["lnZ"] for r in g])
    om = np.mean([r["lnZ"] for r in o])
    sig = math.sqrt(np.mean([r["lnZ_err"] ** 2 for r in g]) / 2 + np.mean([r["lnZ_err"] ** 2 for r in o]) / 2)
    assert abs(gm - om) < 4 * sig, (g, o)
