"""Pins for the oracle's prior-predictive p-value sweep (CPU only).

For y_i ~ N(mu, 1), i = 1..n, mu ~ N(0, lambda^2), the statistic ybar has
prior predictive law N(0, lambda^2 + 1/n), so
    p_lambda = P(|ybar| >= |ybar_obs|) = 2 (1 - Phi(|ybar_obs| / sqrt(lambda^2 + 1/n))).
The oracle's tail-count estimate must match this within Monte Carlo error,
and its data-set means must have that law.
"""
import numpy as np
import pytest
from scipy import stats

import oracle

Z = 4.5


def closed_form_p(lam, ybar_obs, n):
    s = np.sqrt(np.asarray(lam) ** 2 + 1.0 / n)
    return 2.0 * stats.norm.sf(abs(ybar_obs) / s)


@pytest.fixture(scope="module")
def sweep():
    lams = np.array([0.01, 0.3, 1.0, 2.0, 3.0, 10.0, 100.0])
    ybar_obs, n, M = 2.9, 50, 200_000
    counts, p, ybar = oracle.pvalue_sweep(lams, n, M, ybar_obs, seed=2, want_ybar=True)
    return lams, ybar_obs, n, M, counts, p, ybar


def test_p_matches_closed_form(sweep):
    lams, ybar_obs, n, M, counts, p, _ = sweep
    ref = closed_form_p(lams, ybar_obs, n)
    for k in range(lams.size):
        se = np.sqrt(max(ref[k] * (1 - ref[k]), 1e-12) / M)
        assert abs(p[k] - ref[k]) < Z * se + 1.0 / M, (lams[k], p[k], ref[k])
    assert counts[0] == 0  # |ybar_obs| is ~20 prior-predictive sd out at lambda = 0.01
    np.testing.assert_array_equal(p, counts / M)


def test_ybar_has_prior_predictive_law(sweep):
    lams, ybar_obs, n, M, counts, _, ybar = sweep
    for k, lam in enumerate(lams):
        var = lam ** 2 + 1.0 / n
        x = ybar[k]
        assert abs(x.mean()) < Z * np.sqrt(var / M)
        assert abs(x.var() - var) < Z * var * np.sqrt(2.0 / M)
        assert stats.kstest(x[:50_000] / np.sqrt(var), "norm").pvalue > 1e-4
        assert counts[k] == np.count_nonzero(np.abs(x) >= abs(ybar_obs))


def test_thread_count_and_streams():
    lams = np.array([0.5, 1.5])
    c1, _, y1 = oracle.pvalue_sweep(lams, 10, 5000, 1.0, seed=4, want_ybar=True, n_threads=1)
    c7, _, y7 = oracle.pvalue_sweep(lams, 10, 5000, 1.0, seed=4, want_ybar=True, n_threads=7)
    np.testing.assert_array_equal(c1, c7)
    np.testing.assert_array_equal(y1, y7)
    # each lambda has its own substream: equal lambdas still get different data
    _, _, yy = oracle.pvalue_sweep(np.array([1.0, 1.0]), 10, 1000, 1.0, seed=4, want_ybar=True)
    assert not np.allclose(yy[0], yy[1])
