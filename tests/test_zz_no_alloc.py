"""gwl_loglike_static: the batched likelihood for callers that cannot allocate device memory.

Such callers -- a host whose caching allocator already holds the free device
memory (a raw cudaMalloc may fail there), or a loop that must not block (cudaMalloc
and cudaFree can synchronise the device) -- get the same kernels as gwl_loglike with
the per-call scratch in the library's fixed device array.  The checks: on a fresh
context that only ever calls the static entry point, two calls in a row give
gwl_loglike's results bit for bit (computed on a second context) and agree with the
oracle; the context's device memory and the device's free memory do not change; a
calibrated context works the same way; an oversize batch is refused.  This file is
collected last so that a failure here leaves every other test already run.  It
passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import oracle
from helpers import event, tol
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build

    build.build()


def static_twice(ctx, th):
    """Two gwl_loglike_static calls through the C ABI; the context's and the device's memory before and after."""
    from paper_1909_11873_gb300 import gwl

    L = gwl.lib()
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((th.shape[0],), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    bytes0, free0 = L.gwl_device_bytes(ctx.handle), torch.cuda.mem_get_info()[0]
    for out in outs:
        rc = L.gwl_loglike_static(ctx.handle, th.data_ptr(), th.shape[0], out.data_ptr(), stream)
        assert rc == 0, L.gwl_last_error()
    torch.cuda.synchronize()
    assert L.gwl_sync(ctx.handle) == 0
    bytes1, free1 = L.gwl_device_bytes(ctx.handle), torch.cuda.mem_get_info()[0]
    assert bytes1 == bytes0, (bytes0, bytes1)
    assert free0 - free1 < (1 << 20), (free0, free1)
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_matches_gwl_loglike_twice(precision):
    """Two calls in a row: gwl_loglike's results bit for bit, and the oracle's within the parity bars."""
    from paper_1909_11873_gb300 import gwl

    ev = event("c2")
    th_full = I.proposals(ev, 4096, 21)
    th = torch.from_numpy(I.reduced(th_full, ev.sampling)).cuda()
    ref_ctx = gwl.Context.from_event(ev, precision)
    ref = gwl.loglike(ref_ctx, th).cpu().numpy()
    ctx = gwl.Context.from_event(ev, precision)  # never calls gwl_loglike
    for got in static_twice(ctx, th):
        assert np.array_equal(got, ref)
    idx = np.random.default_rng(5).choice(th_full.shape[0], 64, replace=False)
    want = oracle.loglike(ev, th_full[idx])
    assert np.all(np.abs(got[idx] - want) <= tol(precision, want)), np.abs(got[idx] - want).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_calibrated(precision):
    """The calibration model (ten nodes on three detectors, 71 parameters per row) through the static entry."""
    from paper_1909_11873_gb300 import gwl

    ev = event("c2")
    th_full = I.calibrated_proposals(ev, 2048, 23)
    nodes = I.cal_node_freqs(20.0, 1024.0)
    rows = np.ascontiguousarray(np.concatenate([I.reduced(th_full[:, :11], ev.sampling), th_full[:, 11:]], axis=1))
    th = torch.from_numpy(rows).cuda()
    ref_ctx = gwl.Context.from_event(ev, precision)
    ref_ctx.gwl_set_calibration(nodes)
    ref = gwl.loglike(ref_ctx, th).cpu().numpy()
    ctx = gwl.Context.from_event(ev, precision)
    ctx.gwl_set_calibration(nodes)
    for got in static_twice(ctx, th):
        assert np.array_equal(got, ref)
    idx = np.random.default_rng(6).choice(th_full.shape[0], 32, replace=False)
    want = oracle.loglike_cal(ev, nodes, th_full[idx])
    assert np.all(np.abs(got[idx] - want) <= tol(precision, want)), np.abs(got[idx] - want).max()


def test_static_scratch_rejects_oversize_batch():
    from paper_1909_11873_gb300 import gwl

    ev = event("c2")
    ctx = gwl.Context.from_event(ev, 1)
    B = 1 << 20
    th = torch.zeros((B, 11), dtype=torch.float64, device="cuda")
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    L = gwl.lib()
    rc = L.gwl_loglike_static(ctx.handle, th.data_ptr(), B, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"fixed device array" in L.gwl_last_error()
