"""Pins for the oracle's weak-informativity test (Algorithm 2), CPU only.

For the conjugate model with base hyperparameter lambda_0, the p-value of a
base data set under lambda is p = 2(1 - Phi(|ybar_0| / s_lambda)) with
s^2 = lambda^2 + 1/n and ybar_0 ~ N(0, s_0^2).  Solving
P(p <= gamma) = alpha gives the closed form
    gamma_{lambda,alpha} = 2 (1 - Phi((s_0 / s_lambda) Phi^{-1}(1 - alpha/2))),
which the oracle's Monte Carlo cut-offs must match within their sampling
error (delta method for the alpha quantile plus the binomial error of each
p-value).  lambda = lambda_0 must give gamma = alpha.
"""
import numpy as np
from scipy import stats

import oracle


def closed_form_gamma(lam, lam0, n, alpha):
    s0 = np.sqrt(lam0 ** 2 + 1.0 / n)
    sk = np.sqrt(np.asarray(lam) ** 2 + 1.0 / n)
    return 2 * stats.norm.sf((s0 / sk) * stats.norm.isf(alpha / 2))


def sampling_se(lam, lam0, n, alpha, N):
    s0 = np.sqrt(lam0 ** 2 + 1.0 / n)
    sk = np.sqrt(np.asarray(lam) ** 2 + 1.0 / n)
    q = stats.norm.isf(alpha / 2) * s0                  # (1 - alpha) quantile of |ybar_0|
    f = 2 * stats.norm.pdf(q / s0) / s0                 # density of |ybar_0| there
    se_q = np.sqrt(alpha * (1 - alpha) / N) / f
    dg = 2 * stats.norm.pdf(q / sk) / sk
    g = closed_form_gamma(lam, lam0, n, alpha)
    return np.sqrt((dg * se_q) ** 2 + g * (1 - g) / N)


def test_cutoffs_match_closed_form():
    lam = np.array([0.1, 0.5, 1.0, 2.0, 5.0, 20.0])
    lam0, n, N = 1.0, 50, 3000
    for alpha in (0.05, 0.2):
        g, _ = oracle.weakinf(lam, lam0, n, N, alpha, seed=11)
        ref = closed_form_gamma(lam, lam0, n, alpha)
        tol = 4.5 * sampling_se(lam, lam0, n, alpha, N) + 1.0 / N
        assert np.all(np.abs(g - ref) <= tol), (alpha, g, ref, tol)


def test_base_hyperparameter_gives_alpha_and_ordering():
    lam0, n, N, alpha = 2.5, 20, 4000, 0.1
    g, counts = oracle.weakinf(np.array([lam0, 0.5 * lam0, 4 * lam0]), lam0, n, N, alpha,
                               seed=3, want_counts=True)
    se = sampling_se(np.array([lam0]), lam0, n, alpha, N)[0]
    assert abs(g[0] - alpha) <= 4.5 * se + 1.0 / N
    # a narrower prior conflicts more often (smaller cut-off), a wider one less
    assert g[1] < g[0] < g[2]
    # gamma is the ceil(alpha N)-th smallest p-value numerator over N
    r = int(np.ceil(alpha * N))
    for k in range(3):
        assert g[k] == np.sort(counts[k])[r - 1] / N
    assert counts.max() <= N


def test_thread_count_invariance():
    lam = np.array([0.3, 1.0, 3.0, 9.0])
    a, ca = oracle.weakinf(lam, 1.0, 10, 500, 0.05, seed=5, want_counts=True, n_threads=1)
    b, cb = oracle.weakinf(lam, 1.0, 10, 500, 0.05, seed=5, want_counts=True, n_threads=4)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ca, cb)
