"""The launch-shape autotuner (gwl_autotune) and the tuning calls.

The tuned shape must be one of the candidates, the tuned path must still meet
the parity bars against the FP64 oracle, and a bad shape must be refused
without changing the context.
"""
import numpy as np
import pytest

import oracle
from helpers import custom_event, event, tol
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build

    build.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_parity(precision):
    from paper_1909_11873_gb300 import gwl

    ev = event("c2")
    th = I.proposals(ev, 2048, 21)
    ctx = gwl.Context.from_event(ev, precision)
    d = torch.from_numpy(I.reduced(th, ev.sampling)).cuda()
    t = ctx.gwl_autotune(d)
    assert t["window"] % 64 == 0 and 128 <= t["window"] <= 1536
    assert t["grad_window"] % 64 == 0 and 128 <= t["grad_window"] <= 1536
    assert 1 <= t["ctas_per_sm"] <= 4
    assert t["bin_kernel"] in ((gwl.GWL_BINS_WARP, gwl.GWL_BINS_LANE) if precision else (gwl.GWL_BINS_WARP,))
    assert t["ms_loglike"] > 0 and t["ms_grad"] > 0 and t["n_tried"] > 8
    assert ctx.gwl_get_tuning() == t
    idx = np.random.default_rng(3).choice(th.shape[0], 128, replace=False)
    ref = oracle.loglike(ev, th[idx])
    got = gwl.loglike(ctx, d).cpu().numpy()
    assert np.all(np.abs(got[idx] - ref) <= tol(precision, ref))
    lnl, g = gwl.grad(ctx, d[idx])
    assert np.all(np.abs(lnl.cpu().numpy() - ref) <= tol(precision, ref))
    ctx.gwl_sync()


def test_autotune_short_segment_and_bad_shapes():
    """A segment shorter than the smallest window tunes to one window; bad shapes are refused."""
    from paper_1909_11873_gb300 import gwl

    cfg = dict(n_det=2, T=1.0, f_low=20.0, f_high=100.0, noise=True, source="bbh", batch=100, gmst=0.3)
    ev = custom_event(cfg, 8)
    th = I.proposals(ev, 100, 8)
    ctx = gwl.Context.from_event(ev, 1)
    d = torch.from_numpy(I.reduced(th, ev.sampling)).cuda()
    t = ctx.gwl_autotune(d, what=gwl.GWL_TUNE_LOGLIKE)
    assert t["window"] == 128 and t["ms_grad"] == 0.0
    ref = oracle.loglike(ev, th)
    assert np.all(np.abs(gwl.loglike(ctx, d).cpu().numpy() - ref) <= tol(1, ref))
    before = ctx.gwl_get_tuning()
    for bad in (dict(window=100000), dict(window=1000), dict(ctas_per_sm=99), dict(grad_window=-1),
                dict(bin_kernel=4), dict(bin_kernel=-1)):
        with pytest.raises(gwl.GwlError):
            ctx.gwl_set_tuning(**bad)
    assert ctx.gwl_get_tuning() == before
