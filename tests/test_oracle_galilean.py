"""Pins of the oracle's gradient-informed (Galilean) constrained walk, on the CPU.

The walk is a deterministic map of (position, velocity) that preserves volume and undoes itself under
velocity reversal, so the uniform distribution inside the likelihood contour (times the velocity
distribution) is invariant.  The invariance is checked on the analytic Gaussian-in-a-box likelihood,
on a region cut by the cube walls, with an anisotropic step matrix and a periodic coordinate: chains
started uniformly inside the contour must end uniformly inside it, and far from where they started.
The unit-cube gradient that drives the reflections is checked against central differences of the
oracle's likelihood through its prior maps.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import event
from paper_1909_11873_gb300 import inputs as I

scipy_stats = pytest.importorskip("scipy.stats")

MU = np.array([0.1, 0.95, 0.5])
SIGMA = 0.25
RADIUS = 0.3
PERIODIC = np.array([0, 1, 0], dtype=np.int32)
CHOL = np.array([[0.08, 0.0, 0.0], [0.03, 0.05, 0.0], [-0.02, 0.04, 0.06]])


def uniform_in_contour(rng, n):
    """Rejection sample of the cube points with |u - mu| <= RADIUS (the region lnL >= L*)."""
    out = []
    while sum(len(o) for o in out) < n:
        u = rng.uniform(0.0, 1.0, (4 * n, 3))
        out.append(u[np.linalg.norm(u - MU, axis=1) <= RADIUS])
    return np.concatenate(out)[:n]


def lstar():
    return -0.5 * (RADIUS / SIGMA) ** 2 - 3 * math.log(SIGMA * math.sqrt(2 * math.pi))


@pytest.mark.parametrize("persistence", [1.0, 0.5, 0.0])
def test_galilean_walk_keeps_the_constrained_prior_uniform(persistence):
    """Velocity never refreshed, half kept per step, fresh every step."""
    rng = np.random.default_rng(1)
    n, wl = 20000, 40
    u0 = uniform_in_contour(rng, n)
    u1, l1, nacc = oracle.gmc_gauss(MU, SIGMA, PERIODIC, u0, lstar(), seed=7, counter=3, walk_len=wl, scale=1.0,
                                    chol=CHOL, persistence=persistence)
    assert np.all((u1 >= 0.0) & (u1 <= 1.0))
    assert np.all(l1 >= lstar())
    assert np.all(np.linalg.norm(u1 - MU, axis=1) <= RADIUS * (1 + 1e-12))
    assert 0.3 < nacc.mean() / wl < 1.0
    ref = uniform_in_contour(np.random.default_rng(2), 40000)
    for i in range(3):
        assert scipy_stats.ks_2samp(u1[:, i], ref[:, i]).pvalue > 1e-3, i
        assert abs(np.corrcoef(u0[:, i], u1[:, i])[0, 1]) < 0.5, i
    r1, rr = np.linalg.norm(u1 - MU, axis=1), np.linalg.norm(ref - MU, axis=1)
    assert scipy_stats.ks_2samp(r1, rr).pvalue > 1e-3


def test_galilean_walk_is_reproducible_and_moves_only_inside():
    rng = np.random.default_rng(3)
    u0 = uniform_in_contour(rng, 64)
    a = oracle.gmc_gauss(MU, SIGMA, PERIODIC, u0, lstar(), 11, 0, 25, 1.0, CHOL)
    b = oracle.gmc_gauss(MU, SIGMA, PERIODIC, u0, lstar(), 11, 0, 25, 1.0, CHOL, n_threads=1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # a contour no point reaches: every chain stays where it started
    u, l, k = oracle.gmc_gauss(MU, SIGMA, PERIODIC, u0, 1e9, 11, 0, 25, 1.0, CHOL)
    assert np.array_equal(u, u0) and np.all(k == 0)


@pytest.mark.parametrize("name,n_nodes", [("c1", 0), ("c2", 0), ("c1", 4)])
def test_unit_cube_gradient_matches_central_differences(name, n_nodes):
    """d lnL / du through the prior maps (uniform, volume, sine and cosine priors; Gaussian calibration
    priors) against central differences (h = 1e-6) of the oracle's lnL of the mapped point."""
    ev = event(name)
    smp = ev.sampling
    cal = None
    if n_nodes:
        nodes = I.cal_node_freqs(float(ev.freqs[0]), float(ev.freqs[-1]), n_nodes)
        cal = (nodes, 0.1, 0.1)
    Dw = smp.D + (2 * n_nodes * ev.geom.shape[0] if n_nodes else 0)
    rng = np.random.default_rng(4)
    u = rng.uniform(0.05, 0.95, (3, Dw))

    def lnl(pts):
        th = oracle.prior_transform(smp, pts[:, :smp.D])
        if not n_nodes:
            return oracle.loglike(ev, th)
        c = np.arange(Dw - smp.D)
        sg = np.full(c.size, 0.1)
        calp = sg[None, :] * oracle.inv_normal_cdf(pts[:, smp.D:]).reshape(pts.shape[0], -1)
        return oracle.loglike_cal(ev, nodes, np.concatenate([th, calp], axis=1))

    l0, g = oracle.unit_grad(ev, smp, u, cal)
    assert np.allclose(l0, lnl(u), rtol=0, atol=1e-9)
    h = 1e-6
    for k in range(Dw):
        up, um = u.copy(), u.copy()
        up[:, k] += h
        um[:, k] -= h
        fd = (lnl(up) - lnl(um)) / (2 * h)
        assert np.allclose(g[:, k], fd, rtol=1e-5, atol=1e-3 * max(1.0, np.abs(fd).max())), (k, g[:, k], fd)
