"""Device random walks (ns_replace) and nested sampling (ns_run) against the oracle."""
import math

import numpy as np
import pytest

import oracle
from helpers import event
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build
    build.build()


def live_set(ev, K, seed):
    smp = ev.sampling
    u = np.random.default_rng(seed).uniform(0, 1, (K, smp.D))
    ll = oracle.loglike(ev, oracle.prior_transform(smp, u))
    return u, ll


def device_walk(ev, precision, u, ll, worst, lstar, seed, counter, n, walk_len, scale, chol):
    from paper_1909_11873_gb300 import gwl
    ctx = gwl.Context.from_event(ev, precision)
    D = ev.sampling.D
    tu = torch.from_numpy(u).cuda()
    tl = torch.from_numpy(ll).cuda()
    tc = torch.from_numpy(np.ascontiguousarray(chol)).cuda()
    ou = torch.zeros((n, D), dtype=torch.float64, device="cuda")
    ol = torch.zeros(n, dtype=torch.float64, device="cuda")
    on = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.ns_replace(tu, tl, worst, lstar, seed, counter, n, walk_len, scale, tc, ou, ol, on, os_)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    return ou.cpu().numpy(), ol.cpu().numpy(), on.cpu().numpy(), os_.cpu().numpy()


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_ns_replace_replays_oracle_walk_fp64(cfg):
    """Same Philox stream, FP64 likelihood: identical start points and accept counts, end points to 1e-12."""
    ev = event(cfg)
    K = 128
    u, ll = live_set(ev, K, 3)
    worst = int(np.argmin(ll))
    D = ev.sampling.D
    chol = np.diag(np.full(D, 0.04))
    n, wl, seed, ctr = 192, 12, 0x1234ABCD5678, 7
    gu, gl, gn, gs = device_walk(ev, 0, u, ll, worst, ll[worst], seed, ctr, n, wl, 1.0, chol)
    ou, ol, on, os_ = oracle.ns_replace(ev, ev.sampling, u, ll, worst, ll[worst], seed, ctr, n, wl, 1.0, chol)
    assert np.array_equal(gs, os_)
    assert np.array_equal(gn, on)
    assert np.allclose(gu, ou, rtol=0, atol=1e-12)
    assert np.allclose(gl, ol, rtol=0, atol=1e-6)
    assert gn.sum() > 0


def test_ns_replace_mixed_properties():
    """Mixed precision: every chain ends at its start (no accepted step) or at a point whose oracle lnL
    is >= L* within the mixed tolerance and equals the returned lnL within it; acceptance close to FP64's."""
    ev = event("c2")
    K = 128
    u, ll = live_set(ev, K, 4)
    worst = int(np.argmin(ll))
    chol = np.diag(np.full(ev.sampling.D, 0.03))
    n, wl = 256, 10
    gu, gl, gn, gs = device_walk(ev, 1, u, ll, worst, ll[worst], 99, 1, n, wl, 1.0, chol)
    _, _, on, _ = oracle.ns_replace(ev, ev.sampling, u, ll, worst, ll[worst], 99, 1, n, wl, 1.0, chol)
    moved = gn > 0
    assert np.all(gs != worst)
    assert np.allclose(gu[~moved], u[gs[~moved]]) and np.allclose(gl[~moved], ll[gs[~moved]])
    ref = oracle.loglike(ev, oracle.prior_transform(ev.sampling, gu[moved]))
    assert np.all(np.abs(ref - gl[moved]) <= 1e-3)
    assert np.all(ref >= ll[worst] - 1e-3)
    assert abs(gn.mean() - on.mean()) <= 0.05 * max(on.mean(), 1.0)


def test_ns_run_c1_lnz_matches_oracle():
    """Device NS (K = 250, walk length 20) vs the oracle's NS on the zero-noise 1-detector event."""
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    K, nch, wl = 250, 250, 20
    ctx = gwl.Context.from_event(ev, 1)
    g = ctx.ns_run(K, nch, wl, seed=11, dlogz=0.1)
    o = oracle.ns_run(ev, ev.sampling, K, nch, wl, seed=12, dlogz=0.1)
    assert np.isfinite(g["lnZ"]) and g["rounds"] > 3
    sig = math.hypot(g["lnZ_err"], o["lnZ_err"])
    assert abs(g["lnZ"] - o["lnZ"]) < 4 * sig, (g, o)
    # Eq. 5: candidates used per round ~ K ln(1 + n_chains / K)
    assert g["consumed_per_round"] == pytest.approx(K * math.log(1 + nch / K), rel=0.12)


def test_ns_run_posterior_recovers_injection():
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    ctx = gwl.Context.from_event(ev, 1)
    g = ctx.ns_run(200, 200, 20, seed=5, dlogz=0.1, max_dead=20000)
    w = np.exp(g["dead_lnl"] + g["dead_logwt"] - g["lnZ"])
    th = oracle.prior_transform(ev.sampling, g["dead_u"])
    assert abs(np.sum(w * th[:, 0]) / np.sum(w) - 10.0) < 0.05


def test_galilean_walk_properties():
    """Galilean walk: each chain ends at its start or at a point whose oracle lnL >= L* (mixed bar),
    at most one move per step, and it moves at a useful rate."""
    from paper_1909_11873_gb300 import gwl
    ev = event("c2")
    K = 128
    u, ll = live_set(ev, K, 6)
    worst = int(np.argmin(ll))
    D = ev.sampling.D
    ctx = gwl.Context.from_event(ev, 1)
    ctx.gwl_set_walk(gwl.GWL_WALK_GALILEAN)
    n, wl = 256, 10
    tu, tl = torch.from_numpy(u).cuda(), torch.from_numpy(ll).cuda()
    tc = torch.from_numpy(np.diag(np.full(D, 0.03))).cuda()
    ou = torch.zeros((n, D), dtype=torch.float64, device="cuda")
    ol = torch.zeros(n, dtype=torch.float64, device="cuda")
    on = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.ns_replace(tu, tl, worst, ll[worst], 5, 2, n, wl, 1.0, tc, ou, ol, on, os_)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    gu, gl, gn, gs = ou.cpu().numpy(), ol.cpu().numpy(), on.cpu().numpy(), os_.cpu().numpy()
    moved = gn > 0
    assert np.all((gn >= 0) & (gn <= wl)) and moved.mean() > 0.3
    assert np.allclose(gu[~moved], u[gs[~moved]])
    ref = oracle.loglike(ev, oracle.prior_transform(ev.sampling, gu[moved]))
    assert np.all(np.abs(ref - gl[moved]) <= 1e-3)
    assert np.all(ref >= ll[worst] - 1e-3)


def top_live_set(ev, K, seed, n_draw=4096):
    """The K best of n_draw prior points: a live set well inside the prior, so that walks meet the contour."""
    u, ll = live_set(ev, n_draw, seed)
    keep = np.argsort(ll)[-K:]
    return np.ascontiguousarray(u[keep]), np.ascontiguousarray(ll[keep])


@pytest.mark.parametrize("cfg,persistence", [("c1", 1.0), ("c1", 0.5), ("c1", 0.0), ("c2", 0.5)])
def test_galilean_ns_replace_replays_oracle_walk_fp64(cfg, persistence):
    """The Galilean walk against the oracle's (same Philox stream, FP64 likelihood and gradient), with the
    step matrix of the live set's covariance (anisotropic reflections) and a live set that is the best
    128 of 4096 prior points (reflections off the contour and the walls): identical start points and move
    counts, end points to 1e-9."""
    from paper_1909_11873_gb300 import gwl
    ev = event(cfg)
    u, ll = top_live_set(ev, 128, 8)
    worst = int(np.argmin(ll))
    D = ev.sampling.D
    chol = np.linalg.cholesky(np.cov(u.T) + 1e-12 * np.eye(D))
    n, wl, seed, ctr, scale = 96, 12, 0x6A11, 4, 0.5
    ctx = gwl.Context.from_event(ev, 0)
    ctx.gwl_set_walk(gwl.GWL_WALK_GALILEAN)
    ctx.gwl_set_galilean(persistence)
    ou = torch.zeros((n, D), dtype=torch.float64, device="cuda")
    ol = torch.zeros(n, dtype=torch.float64, device="cuda")
    on = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.ns_replace(torch.from_numpy(u).cuda(), torch.from_numpy(ll).cuda(), worst, ll[worst], seed, ctr, n, wl, scale,
                   torch.from_numpy(chol).cuda(), ou, ol, on, os_)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    gu, gl, gn, gs = ou.cpu().numpy(), ol.cpu().numpy(), on.cpu().numpy(), os_.cpu().numpy()
    ru, rl, rn, rs = oracle.gmc_replace(ev, ev.sampling, u, ll, worst, ll[worst], seed, ctr, n, wl, scale, chol,
                                        persistence=persistence)
    assert np.array_equal(gs, rs)
    assert np.array_equal(gn, rn)
    assert np.allclose(gu, ru, rtol=0, atol=1e-9)
    assert np.allclose(gl, rl, rtol=0, atol=1e-6)
    assert 0 < gn.sum() < n * wl  # moves, and some steps that do not move


def test_ns_run_galilean_c1_lnz_matches_oracle():
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    K, nch, wl = 250, 250, 20
    ctx = gwl.Context.from_event(ev, 1)
    ctx.gwl_set_walk(gwl.GWL_WALK_GALILEAN)
    g = ctx.ns_run(K, nch, wl, seed=21, dlogz=0.1)
    o = oracle.ns_run(ev, ev.sampling, K, nch, wl, seed=12, dlogz=0.1)
    sig = math.hypot(g["lnZ_err"], o["lnZ_err"])
    assert abs(g["lnZ"] - o["lnZ"]) < 4 * sig, (g, o)
