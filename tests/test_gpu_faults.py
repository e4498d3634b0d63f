"""Failure detection on the device without a fault (C ABI, gwl_test_wait_timeout and gwl_sync).

The kernels' waits on their bulk copies are bounded by the SM clock: a wait that runs out latches
GWL_ERR_TIMEOUT in the context's status word and the kernel leaves.  Here a kernel waits on a barrier
phase that nothing completes, so the wait runs out by construction; gwl_sync must report the timeout
once and clear it, and the context must keep working.  No test traps, faults or hangs a GPU.
"""
import numpy as np
import pytest

from helpers import event
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build
    build.build()


def test_bounded_wait_timeout_is_latched_reported_and_cleared():
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    ctx = gwl.Context.from_event(ev, gwl.GWL_MIXED)
    th = torch.from_numpy(I.reduced(I.proposals(ev, 64, 3, local_fraction=0.0), ev.sampling)).cuda()
    before = gwl.loglike(ctx, th).cpu().numpy()
    ctx.gwl_sync()
    ctx.gwl_test_wait_timeout(0.05)
    with pytest.raises(gwl.GwlError, match="bounded wait"):
        ctx.gwl_sync()
    ctx.gwl_sync()  # reported once: the latch is cleared
    after = gwl.loglike(ctx, th).cpu().numpy()
    ctx.gwl_sync()
    assert np.array_equal(before, after)
    for bad in (0.0, -1.0, 3.0):
        with pytest.raises(gwl.GwlError):
            ctx.gwl_test_wait_timeout(bad)
