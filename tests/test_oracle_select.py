"""Pins for the oracle's selection and posterior moments (CPU only).

The k-nearest rule (epsilon chosen a posteriori as the k-th smallest
discrepancy) is checked against brute force: numpy's lexicographic sort on
(distance, index) and, on tiny inputs, against enumeration of every subset.
Threshold selection is checked against numpy, epsilon = inf must accept every
sample, and the posterior moments against numpy's mean and var(ddof=1).
"""
import itertools

import numpy as np
import pytest

import oracle


def _brute_topk(d, k):
    order = np.lexsort((np.arange(d.size), d))  # primary key d, then index
    return np.sort(order[:k])


@pytest.mark.parametrize("n", range(1, 9))
def test_topk_matches_subset_enumeration(n):
    rng = np.random.default_rng(n)
    d = rng.choice([0.5, 1.0, 1.5, 2.0], size=n)  # many ties
    for k in range(0, n + 1):
        got = oracle.select_topk(d, k)
        # enumerate every k-subset; keep the one with the smallest sorted
        # (distance, index) key list, which is the tie-broken k nearest.
        best = None
        for sub in itertools.combinations(range(n), k):
            key = sorted((d[i], i) for i in sub)
            if best is None or key < best[0]:
                best = (key, sub)
        np.testing.assert_array_equal(got, np.array(sorted(best[1]), dtype=np.uint64))


def test_topk_matches_numpy_sort_on_large_input():
    rng = np.random.default_rng(0)
    d = rng.gamma(2.0, 1.0, size=100_000)
    d[::97] = d[5]  # forced ties
    for k in (1, 100, 5_000, 99_999, 100_000):
        np.testing.assert_array_equal(oracle.select_topk(d, k), _brute_topk(d, k).astype(np.uint64))


def test_topk_rejects_k_above_n_and_sorts_nan_last():
    with pytest.raises(ValueError):
        oracle.select_topk(np.ones(3), 4)
    d = np.array([np.nan, 3.0, 1.0, np.nan, 2.0])
    np.testing.assert_array_equal(oracle.select_topk(d, 3), [1, 2, 4])
    np.testing.assert_array_equal(oracle.select_topk(d, 4), [0, 1, 2, 4])


def test_threshold_selection():
    rng = np.random.default_rng(1)
    d = rng.uniform(0, 1, size=10_000)
    for eps in (0.0, 0.01, 0.5, 1.0):
        np.testing.assert_array_equal(oracle.select_eps(d, eps), np.nonzero(d <= eps)[0])
    np.testing.assert_array_equal(oracle.select_eps(d, np.inf), np.arange(d.size))


def test_eps_infinity_accepts_every_prior_sample():
    m = {"lo": (0.1, -2, 0.1), "hi": (2, 2, 1), "x0": 0.0, "dt": 0.01, "n_steps": 1000, "n_obs": 10}
    y = np.full(10, 0.5)
    theta, _, dist = oracle.ou_prior_predictive(m, y, 2000, seed=1)
    idx = oracle.select_eps(dist, np.inf)
    assert idx.size == 2000
    mean, var = oracle.moments(theta, idx)
    # with everything accepted the posterior is the prior: U(lo, hi) moments
    lo, hi = np.array(m["lo"]), np.array(m["hi"])
    pm, pv = (lo + hi) / 2, (hi - lo) ** 2 / 12
    assert np.all(np.abs(mean - pm) < 4.5 * np.sqrt(pv / 2000))
    np.testing.assert_allclose(mean, theta.mean(axis=0), rtol=1e-12)


def test_moments_match_numpy():
    rng = np.random.default_rng(2)
    theta = rng.normal(size=(1000, 3)) * [1, 2, 3] + [0.5, -1, 2]
    idx = np.sort(rng.choice(1000, size=137, replace=False)).astype(np.uint64)
    mean, var = oracle.moments(theta, idx)
    sel = theta[idx.astype(np.int64)]
    np.testing.assert_allclose(mean, sel.mean(axis=0), rtol=1e-13)
    np.testing.assert_allclose(var, sel.var(axis=0, ddof=1), rtol=1e-12)
    m1, v1 = oracle.moments(theta, idx[:1])
    np.testing.assert_allclose(m1, theta[int(idx[0])])
    assert np.all(np.isnan(v1))
    m0, v0 = oracle.moments(theta, idx[:0])
    assert np.all(np.isnan(m0)) and np.all(np.isnan(v0))
