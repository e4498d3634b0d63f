"""The device gradient with the calibration model (gwl_grad on a calibrated context) against the oracle.

The row of theta holds the sampled source coordinates and then, per detector, the amplitude and phase
corrections at the nodes; the gradient has the same layout.  The source directions come from the
likelihood's gradient bin loop with the calibration factor applied bin by bin; the calibration
directions from per-interval moments of the spline weights folded through the natural-spline matrix.
The oracle differentiates its calibrated likelihood with dual numbers (oracle.grad_cal).  Scaled errors:
|dg| x width / max(1, |g| x width), width the prior range of a source coordinate, 0.1 (the prior width)
for a calibration coordinate.  Bars: FP64 1e-6; mixed 1e-3 for the calibration directions and, for the
source directions, 1e-3 at the 99th percentile of rows and 1e-2 at the maximum (the FP32 tangents of
the spin directions; see the plain gradient's tests).
"""
import math

import numpy as np
import pytest

import oracle
from helpers import custom_event, event
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CAL_W = 0.1


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build
    build.build()


def nodes_for(ev, n=I.CAL_NODES):
    return I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1]), n)


def run(ev, th, cal, nodes, precision, **tuning):
    from paper_1909_11873_gb300 import gwl
    ctx = gwl.Context.from_event(ev, precision)
    ctx.gwl_set_calibration(nodes)
    if tuning:
        ctx.gwl_set_tuning(**tuning)
    rows = np.ascontiguousarray(np.concatenate([I.reduced(th, ev.sampling), cal], axis=1))
    lnl, g = gwl.grad(ctx, torch.from_numpy(rows).cuda())
    torch.cuda.synchronize()
    ctx.gwl_sync()
    return lnl.cpu().numpy(), g.cpu().numpy()


def scaled_errors(ev, g, ref_g):
    D = ev.sampling.D
    ref_src = ref_g[:, ev.sampling.param_map]
    width = ev.sampling.hi - ev.sampling.lo
    es = np.abs(g[:, :D] - ref_src) * width / np.maximum(np.abs(ref_src) * width, 1.0)
    ec = np.abs(g[:, D:] - ref_g[:, 11:]) * CAL_W / np.maximum(np.abs(ref_g[:, 11:]) * CAL_W, 1.0)
    return es, ec


def check(precision, lnl, ref_l, es, ec):
    if precision == 0:
        assert np.abs(lnl - ref_l).max() <= 1e-6
        assert es.max() <= 1e-6 and ec.max() <= 1e-6, (es.max(), ec.max())
    else:
        assert np.abs(lnl - ref_l).max() <= 1e-3
        assert ec.max() <= 1e-3, ec.max()
        assert np.percentile(es.max(axis=1), 99) <= 1e-3 and es.max() <= 1e-2, (np.percentile(es.max(axis=1), 99), es.max())


@pytest.mark.parametrize("precision", [0, 1])
def test_cal_grad_c1_matches_oracle(precision):
    """1 detector, 4 s, 4 source + 20 calibration coordinates (ten nodes); the cuts span two 640-bin windows."""
    ev = event("c1")
    th = I.proposals(ev, 512, 6, local_fraction=0.5)
    nodes = nodes_for(ev)
    cal = I.draw_calibration(np.random.default_rng(5), 512, 1)
    lnl, g = run(ev, th, cal, nodes, precision)
    idx = np.random.default_rng(1).choice(512, 256, replace=False)
    ref_l, ref_g = oracle.grad_cal(ev, nodes, np.concatenate([th, cal], axis=1)[idx])
    es, ec = scaled_errors(ev, g[idx], ref_g)
    check(precision, lnl[idx], ref_l, es, ec)


@pytest.mark.parametrize("precision", [0, 1])
def test_cal_grad_c2_71d_matches_oracle(precision):
    """3 detectors, 8 s, 11 source + 60 calibration coordinates (71-D), 2048 proposals; 192 rows checked."""
    ev = event("c2")
    th = I.proposals(ev, 2048, 7)
    nodes = nodes_for(ev)
    cal = I.draw_calibration(np.random.default_rng(8), 2048, 3)
    lnl, g = run(ev, th, cal, nodes, precision)
    idx = np.random.default_rng(2).choice(2048, 192, replace=False)
    ref_l, ref_g = oracle.grad_cal(ev, nodes, np.concatenate([th, cal], axis=1)[idx])
    es, ec = scaled_errors(ev, g[idx], ref_g)
    check(precision, lnl[idx], ref_l, es, ec)


@pytest.mark.parametrize("precision", [0, 1])
def test_cal_grad_many_windows_and_short_intervals(precision):
    """3001 bins in 128-bin gradient windows (proposals over up to 24 windows, spline intervals straddling
    windows and 32-bin blocks) with 16 nodes over a 20-395 Hz band, band-mode cut (every bin in band)."""
    cfg = dict(n_det=2, T=8.0, f_low=20.0, f_high=395.0, noise=True, source="bbh", batch=96, gmst=0.9)
    ev = custom_event(cfg, 12, fcut_mode=1)
    th = I.proposals(ev, 96, 12)
    nodes = I.cal_node_freqs(20.0, 395.0, 16)
    cal = I.draw_calibration(np.random.default_rng(13), 96, 2, n_nodes=16)
    lnl, g = run(ev, th, cal, nodes, precision, grad_window=128)
    ref_l, ref_g = oracle.grad_cal(ev, nodes, np.concatenate([th, cal], axis=1))
    es, ec = scaled_errors(ev, g, ref_g)
    check(precision, lnl, ref_l, es, ec)


def test_cal_grad_matches_central_differences_of_device_lnl():
    """The calibration directions against central differences (h = 1e-6) of the FP64 device likelihood."""
    from paper_1909_11873_gb300 import gwl
    ev = event("c2")
    nodes = nodes_for(ev)
    th = I.proposals(ev, 4, 3)
    cal = I.draw_calibration(np.random.default_rng(4), 4, 3)
    _, g = run(ev, th, cal, nodes, 0)
    ctx = gwl.Context.from_event(ev, 0)
    ctx.gwl_set_calibration(nodes)
    rows = np.concatenate([I.reduced(th, ev.sampling), cal], axis=1)
    D = ev.sampling.D
    for b in range(4):
        ks = D + np.arange(0, rows.shape[1] - D, 7)
        pts = []
        for k in ks:
            for s in (1, -1):
                r = rows[b].copy()
                r[k] += s * 1e-6
                pts.append(r)
        l = gwl.loglike(ctx, torch.from_numpy(np.array(pts)).cuda()).cpu().numpy()
        fd = (l[0::2] - l[1::2]) / 2e-6
        assert np.allclose(fd, g[b, ks], rtol=1e-4, atol=1e-3), (b, fd, g[b, ks])


def test_galilean_ns_replace_with_calibration_replays_oracle_walk_fp64():
    """The Galilean walk over 4 source + 8 calibration coordinates against the oracle's (FP64, same stream,
    anisotropic step matrix, live set = best 128 of 2048 prior points): identical start points and move
    counts, end points to 1e-9."""
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    nodes = nodes_for(ev, 4)
    smp = ev.sampling
    Dw = smp.D + 8
    u = np.random.default_rng(6).uniform(0, 1, (2048, Dw))
    cal = 0.1 * oracle.inv_normal_cdf(u[:, smp.D:]).reshape(2048, 8)
    ll = oracle.loglike_cal(ev, nodes, np.concatenate([oracle.prior_transform(smp, u[:, :smp.D]), cal], axis=1))
    keep = np.argsort(ll)[-128:]
    u, ll = np.ascontiguousarray(u[keep]), np.ascontiguousarray(ll[keep])
    worst = int(np.argmin(ll))
    chol = np.linalg.cholesky(np.cov(u.T) + 1e-12 * np.eye(Dw))
    n, wl, seed, ctr, scale = 64, 10, 0xCA1, 2, 0.5
    ctx = gwl.Context.from_event(ev, 0)
    ctx.gwl_set_calibration(nodes, 0.1, 0.1)
    ctx.gwl_set_walk(gwl.GWL_WALK_GALILEAN)
    ou = torch.zeros((n, Dw), dtype=torch.float64, device="cuda")
    ol = torch.zeros(n, dtype=torch.float64, device="cuda")
    on = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.ns_replace(torch.from_numpy(u).cuda(), torch.from_numpy(ll).cuda(), worst, ll[worst], seed, ctr, n, wl, scale,
                   torch.from_numpy(chol).cuda(), ou, ol, on, os_)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    gu, gl, gn, gs = ou.cpu().numpy(), ol.cpu().numpy(), on.cpu().numpy(), os_.cpu().numpy()
    ru, rl, rn, rs = oracle.gmc_replace(ev, smp, u, ll, worst, ll[worst], seed, ctr, n, wl, scale, chol,
                                        cal=(nodes, 0.1, 0.1))
    assert np.array_equal(gs, rs)
    assert np.array_equal(gn, rn)
    assert np.allclose(gu, ru, rtol=0, atol=1e-9)
    assert np.allclose(gl, rl, rtol=0, atol=1e-6)
    assert 0 < gn.sum() < n * wl


def test_galilean_ns_with_calibration_lnz_matches_oracle():
    """The gradient-informed walk over 4 source + 8 calibration coordinates (it needs the calibrated
    gradient): device NS (mixed) against the oracle's random-walk NS of the same posterior; mean lnZ of two
    runs on each side (the calibration phase is degenerate with phi_c, see the random-walk test)."""
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    nodes = nodes_for(ev, 4)
    K, nch, wl = 250, 250, 30
    ctx = gwl.Context.from_event(ev, 1)
    ctx.gwl_set_calibration(nodes, 0.1, 0.1)
    ctx.gwl_set_walk(gwl.GWL_WALK_GALILEAN)
    g = [ctx.ns_run(K, nch, wl, seed=s, dlogz=0.1, max_dead=20000) for s in (31, 33)]
    o = [oracle.ns_run_cal(ev, ev.sampling, (nodes, 0.1, 0.1), K, nch, 60, seed=s, dlogz=0.1) for s in (22, 24)]
    for r in g:
        assert np.isfinite(r["lnZ"]) and r["rounds"] > 3 and r["acceptance"] > 0.0
        assert r["dead_u"].shape[1] == 12
    gm = np.mean([r["lnZ"] for r in g])
    om = np.mean([r["lnZ"] for r in o])
    sig = math.sqrt(np.mean([r["lnZ_err"] ** 2 for r in g]) / 2 + np.mean([r["lnZ_err"] ** 2 for r in o]) / 2)
    assert abs(gm - om) < 4 * sig, (g, o)


def test_autotune_gradient_window_with_calibration():
    """gwl_autotune times gwl_grad on a calibrated batch (windows whose calibration scratch fits) and the
    chosen window gives the same gradient as the default one within the mixed bars."""
    from paper_1909_11873_gb300 import gwl
    ev = event("c2")
    nodes = nodes_for(ev)
    th = I.proposals(ev, 1024, 9)
    cal = I.draw_calibration(np.random.default_rng(10), 1024, 3)
    rows = torch.from_numpy(np.ascontiguousarray(np.concatenate([I.reduced(th, ev.sampling), cal], axis=1))).cuda()
    ctx = gwl.Context.from_event(ev, 1)
    ctx.gwl_set_calibration(nodes)
    l0, g0 = gwl.grad(ctx, rows)
    t = ctx.gwl_autotune(rows, gwl.GWL_TUNE_GRAD)
    assert t["grad_window"] >= 32 and t["ms_grad"] > 0.0
    l1, g1 = gwl.grad(ctx, rows)
    ctx.gwl_sync()
    assert torch.allclose(l0, l1, rtol=0, atol=1e-3)
    width = np.concatenate([ev.sampling.hi - ev.sampling.lo, np.full(rows.shape[1] - ev.sampling.D, CAL_W)])
    a, b = g0.cpu().numpy() * width, g1.cpu().numpy() * width
    err = np.abs(a - b) / np.maximum(np.abs(a), 1.0)
    assert np.percentile(err.max(axis=1), 99) <= 1e-3 and err.max() <= 1e-2
