"""Two and four detectors (four is the library's maximum, GWL_MAX_DET; three are covered by the
configuration tests): parity of the device likelihood (both precisions, one window and several,
with and without the calibration model) and of the gradient with the FP64 oracle.  4 s of data,
20-512 Hz (1969 bins), 256 proposals."""
import numpy as np
import pytest

import oracle
from helpers import custom_event, tol
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CFG = dict(T=4.0, f_low=20.0, f_high=512.0, noise=True, source="bbh", batch=256, gmst=0.7)
GTOL = {0: 1e-6, 1: 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build
    build.build()


@pytest.fixture(scope="module", params=[2, 4], ids=["2det", "4det"])
def ev(request):
    e = custom_event(dict(CFG, n_det=request.param), 21)
    assert e.geom.shape[0] == request.param
    return e


def context(ev, precision, **tuning):
    from paper_1909_11873_gb300 import gwl
    ctx = gwl.Context.from_event(ev, precision)
    if tuning:
        ctx.gwl_set_tuning(**tuning)
    return ctx


@pytest.mark.parametrize("precision", [0, 1])
def test_four_detector_loglike(ev, precision):
    from paper_1909_11873_gb300 import gwl
    th = I.proposals(ev, 256, 4)
    ref = oracle.loglike(ev, th)
    x = torch.from_numpy(I.reduced(th, ev.sampling)).cuda()
    for tuning in ({}, dict(window=128, ctas_per_sm=2)):
        ctx = context(ev, precision, **tuning)
        got = gwl.loglike(ctx, x).cpu().numpy()
        ctx.gwl_sync()
        assert np.all(np.abs(got - ref) <= tol(precision, ref)), (tuning, np.abs(got - ref).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_four_detector_calibrated_loglike(ev, precision):
    from paper_1909_11873_gb300 import gwl
    th = I.proposals(ev, 256, 5)
    nodes = I.cal_node_freqs(20.0, 512.0)
    cal = I.draw_calibration(np.random.default_rng(6), 256, ev.geom.shape[0])
    ref = oracle.loglike_cal(ev, nodes, np.concatenate([th, cal], axis=1))
    rows = np.ascontiguousarray(np.concatenate([I.reduced(th, ev.sampling), cal], axis=1))
    ctx = context(ev, precision)
    ctx.gwl_set_calibration(nodes)
    got = gwl.loglike(ctx, torch.from_numpy(rows).cuda()).cpu().numpy()
    ctx.gwl_sync()
    assert np.all(np.abs(got - ref) <= tol(precision, ref)), np.abs(got - ref).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_four_detector_gradient(ev, precision):
    from paper_1909_11873_gb300 import gwl
    th = I.proposals(ev, 256, 7)
    ctx = context(ev, precision)
    lnl, g = gwl.grad(ctx, torch.from_numpy(I.reduced(th, ev.sampling)).cuda())
    ctx.gwl_sync()
    lnl, g = lnl.cpu().numpy(), g.cpu().numpy()
    idx = np.arange(0, 256, 4)
    ref_l, ref_g = oracle.grad(ev, th[idx])
    assert np.all(np.abs(lnl[idx] - ref_l) <= tol(precision, ref_l))
    width = ev.sampling.hi - ev.sampling.lo
    s = np.maximum(np.abs(ref_g) * width, 1.0)
    err = np.abs(g[idx] - ref_g) * width / s
    assert err.max() <= GTOL[precision], f"max scaled error {err.max():.3e}"
