"""Parity of the device log-likelihood (C ABI, gwl_loglike) with the FP64 oracle.

Bars: |dlnL| <= 1e-6 for GWL_FP64 and <= 1e-3 for GWL_MIXED, absolute at every
|lnL|.  Full batches are compared element by element where the oracle
finishes in seconds, sampled rows otherwise; the same launch configuration
as the benchmark is used.
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


def run_gpu(ev, theta_full, precision, ctx=None, **tuning):
    g = gwl()
    ctx = ctx or g.Context.from_event(ev, precision)
    if tuning:
        ctx.gwl_set_tuning(**tuning)
    th = torch.from_numpy(I.reduced(theta_full, ev.sampling)).cuda()
    out = g.loglike(ctx, th)
    torch.cuda.synchronize()
    ctx.gwl_sync()
    return out.cpu().numpy()


def report(got, ref, precision):
    err = np.abs(got - ref)
    bad = err > tol(precision, ref)
    return f"max |d| = {err.max():.3e}, failing {bad.sum()} / {err.size}"


@pytest.mark.parametrize("precision", [0, 1])
def test_c1_full_batch(precision):
    ev = event("c1")
    th = I.proposals(ev, 1024, 1, local_fraction=0.0)
    ref = oracle.loglike(ev, th)
    got = run_gpu(ev, th, precision)
    assert np.all(np.abs(got - ref) <= tol(precision, ref)), report(got, ref, precision)


@pytest.mark.parametrize("precision,bin_kernel", [(0, 1), (1, 2), (1, 3)])
def test_c2_full_batch_sampled(precision, bin_kernel):
    """8192 proposals (half prior draws, half near the injection) on the device; 384 rows checked; the mixed
    path with both bin-loop layouts (one proposal per warp, one per lane)."""
    ev = event("c2")
    th = I.proposals(ev, 8192, 2)
    got = run_gpu(ev, th, precision, bin_kernel=bin_kernel)
    idx = np.random.default_rng(0).choice(th.shape[0], 384, replace=False)
    ref = oracle.loglike(ev, th[idx])
    assert np.all(np.abs(got[idx] - ref) <= tol(precision, ref)), report(got[idx], ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_c3_long_segment_sampled(precision):
    """128 s, 259,585 bins per detector, 2048 proposals; 256 rows checked (phase up to ~1e4 cycles).

    A BNS chirp spends ~150 s above 20 Hz, so below ~28 Hz a 32-bin block (0.25 Hz) spans more than 16
    cycles of phase and the mixed path forms its deltas in float-float arithmetic: the test checks that
    these blocks ran (a device counter) on every proposal with an in-band bin."""
    g = gwl()
    ev = event("c3")
    th = I.proposals(ev, 2048, 3)
    ctx = g.Context.from_event(ev, precision)
    if precision == 1:
        ctx.gwl_test_ffdelta_blocks(1)
    got = run_gpu(ev, th, precision, ctx=ctx)
    if precision == 1:
        blocks = ctx.gwl_test_ffdelta_blocks(0)
        assert blocks >= 16 * th.shape[0], blocks
    idx = np.random.default_rng(1).choice(th.shape[0], 256, replace=False)
    ref = oracle.loglike(ev, th[idx])
    assert np.all(np.abs(got[idx] - ref) <= tol(precision, ref)), report(got[idx], ref, precision)


@pytest.mark.parametrize("precision,bin_kernel", [(0, 1), (1, 2), (1, 3)])
@pytest.mark.parametrize("fcut_mode", [0, 1])
def test_several_windows_and_ragged_tails(precision, bin_kernel, fcut_mode):
    """3001 bins in windows of 992, 512 and 128 bins, 333 proposals (ragged everywhere); the mixed path with
    both bin-loop layouts (with one proposal per lane: chunks of one window at 992 bins, of 64 bins below)."""
    cfg = dict(n_det=3, T=8.0, f_low=20.0, f_high=395.0, noise=True, source="bbh", batch=333, gmst=0.9)
    ev = custom_event(cfg, 5, fcut_mode=fcut_mode)
    th = I.proposals(ev, 333, 5)
    ref = oracle.loglike(ev, th)
    for window, ctas in ((992, 3), (512, 2), (128, 4)):
        got = run_gpu(ev, th, precision, window=window, ctas_per_sm=ctas, bin_kernel=bin_kernel)
        assert np.all(np.abs(got - ref) <= tol(precision, ref)), report(got, ref, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_edge_rows(precision):
    """Unphysical rows give -inf; a cut below the first bin gives 0; B = 1 works; B = 0 is a no-op."""
    ev = event("c2")
    base = ev.theta_inj.copy()
    rows = np.tile(base, (7, 1))
    rows[1, 1] = 1.2        # q > 1
    rows[2, 0] = -3.0       # Mc < 0
    rows[3, 4] = 0.0        # dL = 0
    rows[4, 6] = np.nan     # non-finite
    rows[5, 0] = 400.0      # f_ISCO below 20 Hz: no bins
    rows[6, 1] = 1.0        # equal masses
    ref = oracle.loglike(ev, rows)
    got = run_gpu(ev, rows, precision)
    assert np.all(np.isneginf(got[1:5]))
    assert got[5] == 0.0 and ref[5] == 0.0
    ok = [0, 6]
    assert np.all(np.abs(got[ok] - ref[ok]) <= tol(precision, ref[ok]))
    one = run_gpu(ev, rows[:1], precision)
    assert abs(one[0] - ref[0]) <= tol(precision, ref[:1])[0]
    g = gwl()
    ctx = g.Context.from_event(ev, precision)
    empty = torch.zeros((0, 11), dtype=torch.float64, device="cuda")
    ctx.gwl_loglike(empty, torch.zeros(0, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", [0, 1])
def test_cut_next_to_bin_frequencies(precision):
    """ISCO cut frequencies 1e-8 and 1e-6 bin widths either side of bin frequencies (q = 1, so
    M = 1 / (6^{3/2} pi T_sun f_cut)): the device's bin count, taken from the grid where the cut is
    more than 1e-7 bins from a bin and settled against the stored frequencies otherwise, must match
    the oracle's per-bin comparison -- one bin more or less moves lnL by that bin's term."""
    ev = event("c2")
    tsun = 4.925490947e-6
    rows, offs = [], (-1e-6, -1e-8, 1e-8, 1e-6)
    for j in (180, 333, 512, 601):
        for d in offs:
            fc = ev.freqs[j] + d * (ev.freqs[1] - ev.freqs[0])
            m = 1.0 / (6.0 ** 1.5 * np.pi * tsun * fc)
            r = ev.theta_inj.copy()
            r[1] = 1.0
            r[0] = m * 0.25 ** 0.6
            rows.append(r)
    rows = np.array(rows)
    ref = oracle.loglike(ev, rows)
    got = run_gpu(ev, rows, precision)
    assert np.all(np.abs(got - ref) <= tol(precision, ref)), report(got, ref, precision)
    # the offsets straddle a bin: the oracle's lnL steps there by much more than the bar
    step = np.abs(ref.reshape(4, 4)[:, 2] - ref.reshape(4, 4)[:, 1])
    assert np.all(step > 100 * tol(precision, ref.reshape(4, 4)[:, 1])), step


@pytest.mark.parametrize("precision,bin_kernel", [(0, 1), (1, 2), (1, 3)])
def test_deterministic_and_host_entry(precision, bin_kernel):
    """Repeated calls are bit-identical: with one proposal per lane the bucket order (and so which
    proposals share a warp) changes from call to call, but every proposal's own arithmetic does not."""
    ev = event("c2")
    th = I.proposals(ev, 3000, 9)
    g = gwl()
    ctx = g.Context.from_event(ev, precision)
    ctx.gwl_set_tuning(bin_kernel=bin_kernel)
    a = run_gpu(ev, th, precision, ctx=ctx)
    b = run_gpu(ev, th, precision, ctx=ctx)
    assert np.array_equal(a, b)
    out = np.zeros(th.shape[0])
    ctx.gwl_loglike_host(np.ascontiguousarray(I.reduced(th, ev.sampling)), out)
    assert np.array_equal(a, out)


def test_waveform_matches_oracle():
    """The device template h_d(f_j) (FP64) agrees with the oracle's per-bin definition."""
    ev = event("c2")
    th = I.proposals(ev, 4, 11)
    g = gwl()
    ctx = g.Context.from_event(ev, 0)
    h = g.waveform(ctx, torch.from_numpy(I.reduced(th, ev.sampling)).cuda()).cpu().numpy()
    for b in range(th.shape[0]):
        ref = oracle.waveform(ev, th[b])
        got = h[b, ..., 0] + 1j * h[b, ..., 1]
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", [0, 1])
def test_host_entry_point_pinned_and_pageable(precision):
    """gwl_loglike_host gives the device entry point's results bit for bit, with page-locked buffers (read
    and written in place by the kernels), pageable buffers (staged) and a mix of the two."""
    g = gwl()
    ev = event("c2")
    rows = np.ascontiguousarray(I.reduced(I.proposals(ev, 3000, 8), ev.sampling))
    ctx = g.Context.from_event(ev, precision)
    ref = g.loglike(ctx, torch.from_numpy(rows).cuda()).cpu().numpy()
    pin_t = torch.from_numpy(rows).pin_memory().numpy()
    pin_l = torch.zeros(3000, dtype=torch.float64).pin_memory().numpy()
    page_l = np.zeros(3000)
    for t, l in ((pin_t, pin_l), (rows, page_l), (pin_t, page_l), (rows, pin_l)):
        l[:] = 0.0
        ctx.gwl_loglike_host(t, l)
        assert np.array_equal(l, ref)


@pytest.mark.parametrize("name,B,rows", [("c1", 1024, 1024), ("c2", 8192, 256), ("c3", 2048, 64)])
def test_fp64_phase_mixed_arm(name, B, rows):
    """GWL_MIXED_F64PHASE -- the phase in FP64 per bin and detector, reduced exactly, then FP32 sine, cosine
    and sums -- against the oracle within the mixed bar, on the three lnL workloads."""
    g = gwl()
    ev = event(name)
    th = I.proposals(ev, B, 4, local_fraction=0.0 if name == "c1" else 0.5)
    got = run_gpu(ev, th, g.GWL_MIXED_F64PHASE)
    idx = np.random.default_rng(7).choice(B, rows, replace=False) if rows < B else np.arange(B)
    ref = oracle.loglike(ev, th[idx])
    assert np.all(np.abs(got[idx] - ref) <= tol(1, ref)), report(got[idx], ref, 1)


def test_fp64_phase_mixed_arm_windows_and_refusals():
    """Several windows with ragged tails; the entry points outside the likelihood refuse the mode."""
    g = gwl()
    cfg = dict(n_det=3, T=8.0, f_low=20.0, f_high=395.0, noise=True, source="bbh", batch=333, gmst=0.9)
    ev = custom_event(cfg, 5)
    th = I.proposals(ev, 333, 5)
    ref = oracle.loglike(ev, th)
    for window, ctas in ((992, 3), (128, 2)):
        got = run_gpu(ev, th, g.GWL_MIXED_F64PHASE, window=window, ctas_per_sm=ctas)
        assert np.all(np.abs(got - ref) <= tol(1, ref)), report(got, ref, 1)
    ctx = g.Context.from_event(ev, g.GWL_MIXED_F64PHASE)
    x = torch.from_numpy(I.reduced(th[:8], ev.sampling)).cuda()
    with pytest.raises(g.GwlError):
        g.grad(ctx, x)
    with pytest.raises(g.GwlError):
        ctx.gwl_set_calibration(I.cal_node_freqs(20.0, 395.0))
    with pytest.raises(g.GwlError):
        g.MultiContext([ctx])
