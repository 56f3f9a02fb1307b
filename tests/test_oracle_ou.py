"""Pins for the oracle's OU prior-predictive sampler (CPU only).

With theta fixed (a degenerate prior lo = hi), the Euler-Maruyama recursion
X_s = a X_{s-1} + th1 th2 dt + th3 sqrt(dt) xi, a = 1 - th1 dt, has the exact
discrete moments
    E[X_s]   = th2 + (x0 - th2) a^s,
    Var[X_s] = th3^2 dt (1 - a^{2s}) / (1 - a^2),
    Cov[X_s, X_t] = a^{t-s} Var[X_s]  (t >= s),
which the oracle's summaries must match within Monte Carlo error.  A wrong
observation step, a dropped sqrt(dt), a sign error in the drift or reused
normals each fail one of these checks.  The prior draws, the Euclidean
discrepancy and the counter keying are pinned separately.
"""
import numpy as np
import pytest
from scipy import stats

import oracle

Z = 4.5  # standard errors allowed


def _fixed_model(theta, dt, n_steps, n_obs, x0):
    return {"lo": theta, "hi": theta, "x0": x0, "dt": dt, "n_steps": n_steps, "n_obs": n_obs}


@pytest.fixture(scope="module")
def fixed_paths():
    theta = (2.0, 0.5, 0.8)
    dt, S, n_obs, x0 = 0.05, 40, 10, 0.7
    m = _fixed_model(theta, dt, S, n_obs, x0)
    y = np.zeros(n_obs)
    _, summ, dist = oracle.ou_prior_predictive(m, y, 200_000, seed=77, want_theta=False,
                                                want_summ=True)
    return theta, dt, S, n_obs, x0, summ, dist


def test_discrete_em_mean_and_variance(fixed_paths):
    (th1, th2, th3), dt, S, n_obs, x0, summ, _ = fixed_paths
    a = 1.0 - th1 * dt
    N = summ.shape[0]
    for j in range(1, n_obs + 1):
        s = (j * S) // n_obs
        mean = th2 + (x0 - th2) * a ** s
        var = th3 ** 2 * dt * (1 - a ** (2 * s)) / (1 - a ** 2)
        x = summ[:, j - 1]
        assert abs(x.mean() - mean) < Z * np.sqrt(var / N), (j, x.mean(), mean)
        assert abs(x.var(ddof=1) - var) < Z * var * np.sqrt(2.0 / (N - 1)), (j, x.var(), var)


def test_discrete_em_autocovariance(fixed_paths):
    (th1, th2, th3), dt, S, n_obs, x0, summ, _ = fixed_paths
    a = 1.0 - th1 * dt
    for j in (1, 4, 8):
        s, t = (j * S) // n_obs, ((j + 1) * S) // n_obs
        var_s = th3 ** 2 * dt * (1 - a ** (2 * s)) / (1 - a ** 2)
        var_t = th3 ** 2 * dt * (1 - a ** (2 * t)) / (1 - a ** 2)
        rho = a ** (t - s) * var_s / np.sqrt(var_s * var_t)
        r = np.corrcoef(summ[:, j - 1], summ[:, j])[0, 1]
        # Fisher z standard error
        assert abs(np.arctanh(r) - np.arctanh(rho)) < Z / np.sqrt(summ.shape[0] - 3), (j, r, rho)


def test_observation_steps_with_ragged_division():
    # S = 37 steps, 10 observations: s_j = floor(37 j / 10) = 3, 7, 11, 14, ...
    th1, th2, th3, dt, x0 = 1.5, -0.4, 0.6, 0.04, 1.2
    S, n_obs = 37, 10
    m = _fixed_model((th1, th2, th3), dt, S, n_obs, x0)
    _, summ, _ = oracle.ou_prior_predictive(m, np.zeros(n_obs), 100_000, seed=5,
                                             want_theta=False, want_summ=True)
    a = 1 - th1 * dt
    N = summ.shape[0]
    for j in range(1, n_obs + 1):
        s = (j * S) // n_obs
        mean = th2 + (x0 - th2) * a ** s
        var = th3 ** 2 * dt * (1 - a ** (2 * s)) / (1 - a ** 2)
        assert abs(summ[:, j - 1].mean() - mean) < Z * np.sqrt(var / N), j


def test_small_dt_approaches_continuous_ou():
    # Euler-Maruyama approximates the OU SDE: at dt = 1e-3 the moments at t = 1
    # match the continuous transition within MC error plus an O(dt) allowance.
    th1, th2, th3, x0 = 1.0, 0.5, 0.3, 0.0
    dt, S = 1e-3, 1000
    m = _fixed_model((th1, th2, th3), dt, S, 1, x0)
    _, summ, _ = oracle.ou_prior_predictive(m, np.zeros(1), 40_000, seed=11,
                                             want_theta=False, want_summ=True)
    t = 1.0
    mean = th2 + (x0 - th2) * np.exp(-th1 * t)
    var = th3 ** 2 * (1 - np.exp(-2 * th1 * t)) / (2 * th1)
    x = summ[:, 0]
    N = x.size
    assert abs(x.mean() - mean) < Z * np.sqrt(var / N) + 2 * dt
    assert abs(x.var() - var) < Z * var * np.sqrt(2.0 / N) + 2 * dt * var


def test_prior_draws_are_uniform_on_the_box():
    lo, hi = (0.1, -2.0, 0.1), (2.0, 2.0, 1.0)
    m = {"lo": lo, "hi": hi, "x0": 0.0, "dt": 0.1, "n_steps": 10, "n_obs": 10}
    theta, _, _ = oracle.ou_prior_predictive(m, np.zeros(10), 100_000, seed=3)
    for j in range(3):
        assert theta[:, j].min() > lo[j] and theta[:, j].max() < hi[j]
        assert stats.kstest(theta[:, j], "uniform", args=(lo[j], hi[j] - lo[j])).pvalue > 1e-4
    c = np.corrcoef(theta.T)
    for i in range(3):
        for j in range(i + 1, 3):
            assert abs(c[i, j]) < Z / np.sqrt(theta.shape[0])


def test_distance_is_euclidean_on_the_summaries():
    m = {"lo": (0.1, -2, 0.1), "hi": (2, 2, 1), "x0": 0.0, "dt": 0.05, "n_steps": 200, "n_obs": 10}
    y = np.linspace(-1.0, 1.5, 10)
    _, summ, dist = oracle.ou_prior_predictive(m, y, 5000, seed=9, want_summ=True)
    np.testing.assert_allclose(dist, np.linalg.norm(summ - y[None, :], axis=1), rtol=1e-13)
    # observations enter in order: reversing y changes the distances
    _, _, dist_rev = oracle.ou_prior_predictive(m, y[::-1].copy(), 5000, seed=9)
    assert not np.allclose(dist, dist_rev)


def test_sample_index_keys_the_counter():
    m = {"lo": (0.1, -2, 0.1), "hi": (2, 2, 1), "x0": 0.0, "dt": 0.01, "n_steps": 100, "n_obs": 10}
    y = np.ones(10) * 0.3
    th_full, _, d_full = oracle.ou_prior_predictive(m, y, 3000, seed=21, n_threads=1)
    th_part, _, d_part = oracle.ou_prior_predictive(m, y, 1000, seed=21, base=1500, n_threads=3)
    np.testing.assert_array_equal(d_full[1500:2500], d_part)
    np.testing.assert_array_equal(th_full[1500:2500], th_part)
    _, _, d_t8 = oracle.ou_prior_predictive(m, y, 3000, seed=21, n_threads=8)
    np.testing.assert_array_equal(d_full, d_t8)
    _, _, d_sub = oracle.ou_prior_predictive(m, y, 3000, seed=21, sub=1)
    _, _, d_seed = oracle.ou_prior_predictive(m, y, 3000, seed=22)
    assert not np.allclose(d_full, d_sub) and not np.allclose(d_full, d_seed)


def test_invalid_arguments_are_rejected():
    m = {"lo": (0.1, -2, 0.1), "hi": (2, 2, 1), "x0": 0.0, "dt": 0.01, "n_steps": 5, "n_obs": 10}
    with pytest.raises(ValueError):
        oracle.ou_prior_predictive(m, np.zeros(10), 10, seed=1)      # fewer steps than observations
    m2 = dict(m, n_steps=100, dt=0.0)
    with pytest.raises(ValueError):
        oracle.ou_prior_predictive(m2, np.zeros(10), 10, seed=1)     # dt must be positive
