"""The PP driver's statistics (CPU): Kolmogorov-Smirnov against U(0, 1) and Fisher's combination."""
import numpy as np
import pytest


def test_pp_statistics_helpers():
    """The PP driver's KS statistic equals the textbook sup-distance, and its p-values behave."""
    from paper_1909_11873_gb300.pp_run import fisher, ks_uniform

    rng = np.random.default_rng(5)
    x = rng.uniform(size=200)
    d, p = ks_uniform(x)
    xs = np.sort(x)
    i = np.arange(1, 201)
    assert d == pytest.approx(max(np.max(i / 200 - xs), np.max(xs - (i - 1) / 200)))
    assert p > 0.01
    assert ks_uniform(x ** 2)[1] < 1e-6  # a skewed sample is rejected
    # Fisher: one p-value gives itself back; k equal p-values combine to chi^2_{2k} survival
    assert fisher([0.3]) == pytest.approx(0.3)
    assert fisher([1.0, 1.0]) == pytest.approx(1.0)
