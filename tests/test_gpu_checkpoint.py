"""Checkpoint and resume of the device nested sampler (ns_run_resumable).

The walk's random numbers come from a counter-based generator keyed by the round, and every other part
of a round is a deterministic function of the state carried in a checkpoint, so a run split into calls
must equal one uninterrupted call bit for bit: evidence, information, counts and the dead points."""
import numpy as np
import pytest

from helpers import event
from paper_1909_11873_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KEYS = ("lnZ", "lnZ_err", "H", "n_dead", "n_proposals", "rounds", "scale", "acceptance", "consumed_per_round",
        "dlogz", "n_dead_returned")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build
    build.build()


def same(a, b):
    for k in KEYS:
        assert a[k] == b[k], (k, a[k], b[k])
    for k in ("dead_lnl", "dead_logwt", "dead_u"):
        assert np.array_equal(a[k], b[k]), k


def split_run(ctx, pieces, **kw):
    state = None
    for i, r in enumerate(pieces):
        out = ctx.ns_run(max_rounds=r, resume=state, checkpoint=True, **kw)
        state = out.pop("state")
    return out


def ctx_c1(precision=1, walk=0, cal_nodes=0):
    from paper_1909_11873_gb300 import gwl
    ev = event("c1")
    ctx = gwl.Context.from_event(ev, precision)
    if cal_nodes:
        ctx.gwl_set_calibration(I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1]), cal_nodes), 0.1, 0.1)
    ctx.gwl_set_walk(walk)
    return ctx


@pytest.mark.parametrize("precision", [0, 1])
def test_split_run_equals_uninterrupted(precision):
    kw = dict(K=250, n_chains=250, walk_len=20, seed=11, dlogz=0.1, max_dead=20000)
    ctx = ctx_c1(precision)
    whole = ctx.ns_run(max_rounds=100000, **kw)
    assert whole["rounds"] > 20
    split = split_run(ctx, [7, 6, 100000], **kw)
    same(whole, split)
    # a call that stops early reports the run as if it ended there, and its checkpoint continues it
    part = ctx.ns_run(max_rounds=9, checkpoint=True, **kw)
    assert part["rounds"] == 9 and part["n_dead"] < whole["n_dead"]
    rest = ctx.ns_run(max_rounds=100000, resume=part["state"], **kw)
    same(whole, rest)


@pytest.mark.parametrize("walk,cal_nodes", [(1, 0), (0, 4), (1, 4)])
def test_split_run_galilean_and_calibrated(walk, cal_nodes):
    """The gradient-informed walk (fresh velocities every round) and the calibrated walk dimension."""
    kw = dict(K=200, n_chains=200, walk_len=12, seed=5, dlogz=0.5, max_dead=20000)
    ctx = ctx_c1(1, walk, cal_nodes)
    whole = ctx.ns_run(max_rounds=100000, **kw)
    split = split_run(ctx, [5, 11, 100000], **kw)
    same(whole, split)


def test_checkpointed_npz_file_resumes(tmp_path):
    kw = dict(K=250, n_chains=250, walk_len=20, seed=13, dlogz=0.1, max_dead=20000)
    ctx = ctx_c1(1)
    whole = ctx.ns_run(max_rounds=100000, **kw)
    path = str(tmp_path / "ns_state.npz")
    # an interrupted run: stop after 12 rounds, then a fresh call continues from the file
    first = ctx.ns_run_checkpointed(path, every=4, max_rounds=12, **kw)
    assert first["rounds"] == 12
    out = ctx.ns_run_checkpointed(path, every=4, **kw)
    same(whole, out)


def test_resume_buffer_checks():
    from paper_1909_11873_gb300 import gwl
    kw = dict(n_chains=64, walk_len=4, seed=1, dlogz=0.1, max_dead=0)
    ctx = ctx_c1(1)
    part = ctx.ns_run(K=64, max_rounds=2, checkpoint=True, **kw)
    st = part["state"]
    assert st.size == gwl.lib().ns_state_doubles(64, ctx.theta_stride, 0)
    with pytest.raises(gwl.GwlError, match="another K"):
        ctx.ns_run(K=128, max_rounds=2, resume=np.concatenate([st, np.zeros(1000)]), **kw)
    bad = st.copy()
    bad[0] = 1.0
    with pytest.raises(gwl.GwlError, match="format"):
        ctx.ns_run(K=64, max_rounds=2, resume=bad, **kw)


def test_multi_split_run_equals_uninterrupted():
    """gwl_multi_ns_run_resumable: three events run in three calls through checkpoints give, event by event,
    the uninterrupted run's results exactly; the buffer is checked against the batch and K."""
    from paper_1909_11873_gb300 import gwl
    from test_gpu_multi import four_d, small_events
    evs = [four_d(ev) for ev in small_events()[:3]]
    mc = gwl.MultiContext([gwl.Context.from_event(ev, 1) for ev in evs])
    kw = dict(K=150, n_chains=150, walk_len=16, seed=3, dlogz=0.1)
    whole = mc.gwl_multi_ns_run(max_rounds=100000, **kw)
    assert all(r["rounds"] > 8 for r in whole)
    state = None
    for rounds in (5, 6, 100000):
        out, state = mc.gwl_multi_ns_run(max_rounds=rounds, resume=state, checkpoint=True, **kw)
    for a, b in zip(whole, out):
        for k in KEYS:
            assert a[k] == b[k], (k, a[k], b[k])
    assert state.size == gwl.lib().gwl_multi_ns_state_doubles(mc._h, 150)
    with pytest.raises(gwl.GwlError, match="does not match"):
        mc.gwl_multi_ns_run(K=200, n_chains=150, walk_len=16, seed=3, max_rounds=2,
                            resume=np.concatenate([state, np.zeros(200000)]))
    bad = state.copy()
    bad[0] = 1.0
    with pytest.raises(gwl.GwlError, match="does not match"):
        mc.gwl_multi_ns_run(max_rounds=2, resume=bad, **kw)
