"""gwl_loglike_static: the batched likelihood for callers that cannot allocate device memory.

Such callers (a host whose caching allocator owns the free device memory, or a
loop that must not block on cudaMalloc/cudaFree) get the same kernels as
gwl_loglike with the per-call scratch in the library's fixed device array.
This file is collected last so that a failure here leaves every other test
already run.  It passes alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import event, tol
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build

    build.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_matches_gwl_loglike_twice(precision):
    """Two calls in a row through the C ABI agree with gwl_loglike within the parity tolerance."""
    from paper_1909_11873_gb300 import gwl

    ev = event("c2")
    th = torch.from_numpy(I.reduced(I.proposals(ev, 4096, 21), ev.sampling)).cuda()
    ctx = gwl.Context.from_event(ev, precision)
    L = gwl.lib()
    stream = torch.cuda.current_stream().cuda_stream
    ref = torch.empty(th.shape[0], dtype=torch.float64, device="cuda")
    assert L.gwl_loglike(ctx.handle, th.data_ptr(), th.shape[0], ref.data_ptr(), stream) == 0
    for _ in range(2):
        out = torch.full((th.shape[0],), np.nan, dtype=torch.float64, device="cuda")
        rc = L.gwl_loglike_static(ctx.handle, th.data_ptr(), th.shape[0], out.data_ptr(), stream)
        assert rc == 0, L.gwl_last_error()
        torch.cuda.synchronize()
        assert L.gwl_sync(ctx.handle) == 0
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.abs(o - r) <= tol(precision, r))


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
