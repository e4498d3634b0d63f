"""Parity of the calibrated device log-likelihood (gwl_set_calibration, then
gwl_loglike through the C ABI) with the FP64 oracle's calibration model.

The calibration model of Section 2.2 multiplies each detector's template by
(1 + dA_d(f)) exp(i dphi_d(f)), natural cubic splines in ln f through per-node
corrections.  Bars as for the plain likelihood: |dlnL| <= 1e-6 (GWL_FP64) and
<= 1e-3 (GWL_MIXED), absolute at every |lnL|.
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


def gwl():
    from paper_1909_11873_gb300 import gwl as g

    return g


def cal_context(ev, nodes, precision, **tuning):
    g = gwl()
    ctx = g.Context.from_event(ev, precision)
    ctx.gwl_set_calibration(nodes)
    if tuning:
        ctx.gwl_set_tuning(**tuning)
    return ctx


def device_rows(ev, th_full, cal):
    return np.ascontiguousarray(np.concatenate([I.reduced(th_full, ev.sampling), cal], axis=1))


def run_cal(ev, th_full, cal, nodes, precision, ctx=None, **tuning):
    g = gwl()
    ctx = ctx or cal_context(ev, nodes, precision, **tuning)
    rows = device_rows(ev, th_full, cal)
    assert ctx.theta_stride == rows.shape[1]
    out = g.loglike(ctx, torch.from_numpy(rows).cuda())
    torch.cuda.synchronize()
    ctx.gwl_sync()
    return out.cpu().numpy()


def ref_cal(ev, th_full, cal, nodes):
    return oracle.loglike_cal(ev, nodes, np.concatenate([th_full, cal], axis=1))


def report(got, ref, precision):
    err = np.abs(got - ref)
    bad = err > tol(precision, ref)
    return f"max |d| = {err.max():.3e}, failing {bad.sum()} / {err.size}"


@pytest.mark.parametrize("precision", [0, 1])
def test_c1_full_batch_calibrated(precision):
    """One detector, 1969 bins, 1024 prior draws, ten nodes over the band."""
    ev = event("c1")
    th = I.proposals(ev, 1024, 11, local_fraction=0.0)
    nodes = I.cal_node_freqs(20.0, 512.0)
    cal = I.draw_calibration(np.random.default_rng(3), 1024, 1)
    ref = ref_cal(ev, th, cal, nodes)
    got = run_cal(ev, th, cal, nodes, precision)
    assert np.all(np.abs(got - ref) <= tol(precision, ref)), report(got, ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_c2_calibrated_sampled(precision):
    """3 detectors, 8033 bins, 8192 proposals with 60 calibration parameters (71 per row); 256 rows checked."""
    ev = event("c2")
    th = I.calibrated_proposals(ev, 8192, 2)
    nodes = I.cal_node_freqs(20.0, 1024.0)
    got = run_cal(ev, th[:, :11], th[:, 11:], nodes, precision)
    idx = np.random.default_rng(0).choice(th.shape[0], 256, replace=False)
    ref = oracle.loglike_cal(ev, nodes, th[idx])
    assert np.all(np.abs(got[idx] - ref) <= tol(precision, ref)), report(got[idx], ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("fcut_mode", [0, 1])
def test_calibrated_several_windows_and_ragged_tails(precision, fcut_mode):
    """3001 bins in windows of 832, 512 and 128 bins (several windows per proposal), 333 proposals.
    (832 bins is the largest window of FP64 and calibration rows within shared memory.)"""
    cfg = dict(n_det=3, T=8.0, f_low=20.0, f_high=395.0, noise=True, source="bbh", batch=333, gmst=0.9)
    ev = custom_event(cfg, 5, fcut_mode=fcut_mode)
    th = I.proposals(ev, 333, 5)
    nodes = I.cal_node_freqs(20.0, 395.0)
    cal = I.draw_calibration(np.random.default_rng(4), 333, 3)
    ref = ref_cal(ev, th, cal, nodes)
    for window, ctas in ((832, 3), (512, 2), (128, 4)):
        got = run_cal(ev, th, cal, nodes, precision, window=window, ctas_per_sm=ctas)
        assert np.all(np.abs(got - ref) <= tol(precision, ref)), report(got, ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_calibration_node_layouts(precision):
    """Nodes inside the band (the end cubics continued beyond them), two nodes (a line in ln f)
    and the maximum of sixteen nodes."""
    ev = event("c2")
    th = I.proposals(ev, 200, 7)
    rng = np.random.default_rng(8)
    for nodes in (np.geomspace(45.0, 300.0, 6), np.array([30.0, 700.0]), np.geomspace(20.0, 1024.0, 16)):
        cal = I.draw_calibration(rng, 200, 3, n_nodes=nodes.size)
        ref = ref_cal(ev, th, cal, nodes)
        got = run_cal(ev, th, cal, nodes, precision)
        assert np.all(np.abs(got - ref) <= tol(precision, ref)), report(got, ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_calibration_edge_rows_and_entry_points(precision):
    """Zero corrections give the uncalibrated device result; unphysical rows give -inf; the host and
    static entry points agree; switching calibration off restores the plain row layout."""
    g = gwl()
    ev = event("c2")
    nodes = I.cal_node_freqs(20.0, 1024.0)
    th = np.tile(ev.theta_inj, (6, 1))
    th[1, 1] = 1.2     # q > 1
    th[2, 4] = 0.0     # dL = 0
    th[3, 0] = 400.0   # no in-band bin
    th[4:] = I.proposals(ev, 2, 9)
    cal = I.draw_calibration(np.random.default_rng(5), 6, 3)
    ref = ref_cal(ev, th, cal, nodes)
    ctx = cal_context(ev, nodes, precision)
    got = run_cal(ev, th, cal, nodes, precision, ctx=ctx)
    assert np.all(np.isneginf(got[1:3])) and got[3] == 0.0 and ref[3] == 0.0
    ok = [0, 4, 5]
    assert np.all(np.abs(got[ok] - ref[ok]) <= tol(precision, ref[ok])), report(got[ok], ref[ok], precision)

    rows = device_rows(ev, th, cal)
    host = np.zeros(6)
    ctx.gwl_loglike_host(rows, host)
    assert np.array_equal(np.isneginf(host), np.isneginf(got))
    fin = np.isfinite(got)
    assert np.all(np.abs(host[fin] - got[fin]) <= tol(precision, got[fin]))
    st = torch.empty(6, dtype=torch.float64, device="cuda")
    ctx.gwl_loglike_static(torch.from_numpy(rows).cuda(), st)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert np.all(np.abs(st[fin] - got[fin]) <= tol(precision, got[fin]))

    zero = run_cal(ev, th, np.zeros_like(cal), nodes, precision, ctx=ctx)
    plain_ctx = g.Context.from_event(ev, precision)
    plain = g.loglike(plain_ctx, torch.from_numpy(I.reduced(th, ev.sampling)).cuda()).cpu().numpy()
    assert np.all(np.abs(zero[fin] - plain[fin]) <= tol(precision, plain[fin]))

    ctx.gwl_set_calibration([])
    assert ctx.gwl_get_calibration() == (0, ev.sampling.D)
    off = g.loglike(ctx, torch.from_numpy(I.reduced(th, ev.sampling)).cuda()).cpu().numpy()
    assert np.all(np.abs(off[fin] - plain[fin]) <= tol(precision, plain[fin]))


def test_calibration_refused_where_not_modelled():
    """The FP64-phase arm refuses the model (GWL_ERR_ARG); invalid node sets and prior widths are refused
    (multi-event batches of calibrated contexts: tests/test_gpu_multi.py)."""
    g = gwl()
    ev = event("c2")
    ctx = cal_context(ev, I.cal_node_freqs(20.0, 1024.0), 1)
    f64ph = g.Context.from_event(ev, g.GWL_MIXED_F64PHASE)
    with pytest.raises(g.GwlError):
        f64ph.gwl_set_calibration(I.cal_node_freqs(20.0, 1024.0))
    assert f64ph.gwl_get_calibration()[0] == 0
    for bad in ([20.0], [20.0, 20.0, 30.0], [-1.0, 30.0], np.geomspace(20, 1024, 17)):
        with pytest.raises(g.GwlError):
            ctx.gwl_set_calibration(bad)
    for sa, sp in ((0.0, 0.1), (0.1, -1.0), (np.inf, 0.1)):
        with pytest.raises(g.GwlError):
            ctx.gwl_set_calibration(I.cal_node_freqs(20.0, 1024.0), sa, sp)
    assert ctx.gwl_get_calibration()[0] == 10  # a refused set leaves the context as it was
