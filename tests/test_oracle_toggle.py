"""Pins for the oracle's genetic-toggle-switch prior predictive (CPU only).

* With beta_u = beta_v = 0 the production terms are alpha/2, so (far from the
  clamp) u follows the linear recursion u_j = 0.97 u_{j-1} + alpha_u/2 - 1
  + 0.5 zeta with exact moments, and with gamma = 0 the observation adds an
  independent N(mu, (mu sigma)^2): the mean and variance of y over cells are
  fixed in closed form.
* The coupling direction: a large v represses u (p_u = v^beta_u), a v held
  at the floor does not.
* The floor at 1 (the C listing of Sec. 3.4 clamps u and v after each
  update): with alpha_u = alpha_v = -1000 and beta = 0 every unclamped update
  lands below -400 whatever the normal (|zeta| <= 5.77 for this generator), so
  u = v = 1 exactly after every step, and y = 1 + mu + mu sigma eta is
  N(1 + mu, (mu sigma)^2) for any gamma.  Without the clamp u would end near
  -1.7e4; a clamp at 0, or one applied before the update, ends elsewhere.
* The 19 summaries are numpy's linear-interpolation quantiles of the cells'
  y values, rho is their Euclidean distance to the observed ones, y >= 1,
  and the prior draws are uniform on the paper's box.
"""
import numpy as np
import pytest
from scipy import stats

import oracle

PAPER_LO = (250.0, 0.05, 0.05, 0.0, 0.0, 0.0, 0.0)
PAPER_HI = (400.0, 0.5, 0.35, 50.0, 50.0, 7.0, 7.0)
Z = 4.5


def fixed(theta, T, C):
    return {"lo": tuple(theta), "hi": tuple(theta), "T": T, "C": C}


def _linear_u_moments(alpha, T):
    s, a = T - 1, 0.97
    mean_u = a ** s * 10 + (alpha / 2 - 1) * (1 - a ** s) / (1 - a)
    var_u = 0.25 * (1 - a ** (2 * s)) / (1 - a ** 2)
    return mean_u, var_u


def test_linear_regime_state_moments():
    # sigma ~ 0: y = u + mu, so y's moments are u's (0.97, alpha/2 - 1, 0.5 zeta)
    mu, sigma, alpha = 300.0, 1e-6, 44.0
    T, C, n = 50, 8000, 4
    m = fixed((mu, sigma, 0.3, alpha, alpha, 0.0, 0.0), T, C)
    _, _, y, _ = oracle.toggle_prior_predictive(m, np.zeros(19), n, seed=3, want_y=True)
    y = y.ravel()
    mean_u, var_u = _linear_u_moments(alpha, T)
    N = y.size
    assert abs(y.mean() - (mean_u + mu)) < Z * np.sqrt(var_u / N), (y.mean(), mean_u + mu)
    assert abs(y.var() - var_u) < Z * var_u * np.sqrt(2.0 / N) + 1e-6, (y.var(), var_u)


def test_linear_regime_both_states():
    # beta_u = beta_v = 0: u and v are independent linear recursions (alpha_u, alpha_v differ)
    T, C = 60, 8000
    m = fixed((300.0, 0.1, 0.2, 44.0, 30.0, 0.0, 0.0), T, C)
    *_, uv = oracle.toggle_prior_predictive(m, np.zeros(19), 2, seed=8, want_uv=True)
    for col, alpha in ((0, 44.0), (1, 30.0)):
        x = uv[:, :, col].ravel()
        mean, var = _linear_u_moments(alpha, T)
        assert abs(x.mean() - mean) < Z * np.sqrt(var / x.size), (col, x.mean(), mean)
        assert abs(x.var() - var) < Z * var * np.sqrt(2.0 / x.size), (col, x.var(), var)
    r = np.corrcoef(uv[:, :, 0].ravel(), uv[:, :, 1].ravel())[0, 1]
    assert abs(r) < Z / np.sqrt(uv[:, :, 0].size)  # zeta_u and zeta_v are independent


def test_linear_regime_observation_noise():
    # u is exactly Gaussian here; Var[y] = Var[u] + (mu sigma)^2 E[u^(-2 gamma)]
    mu, sigma, gam, alpha = 300.0, 0.1, 0.3, 44.0
    T, C, n = 50, 8000, 4
    m = fixed((mu, sigma, gam, alpha, alpha, 0.0, 0.0), T, C)
    _, _, y, _ = oracle.toggle_prior_predictive(m, np.zeros(19), n, seed=4, want_y=True)
    y = y.ravel()
    mean_u, var_u = _linear_u_moments(alpha, T)
    x, w = np.polynomial.hermite_e.hermegauss(60)
    e_u = np.sum(w * (mean_u + np.sqrt(var_u) * x) ** (-2 * gam)) / np.sqrt(2 * np.pi)
    var_y = var_u + (mu * sigma) ** 2 * e_u
    N = y.size
    assert abs(y.mean() - (mean_u + mu)) < Z * np.sqrt(var_y / N)
    assert abs(y.var() - var_y) < Z * var_y * np.sqrt(2.0 / N), (y.var(), var_y)


def test_clamp_holds_both_states_at_the_floor():
    mu, sigma, gam = 300.0, 0.05, 0.7
    T, C, n = 40, 8000, 2
    m = fixed((mu, sigma, gam, -1000.0, -1000.0, 0.0, 0.0), T, C)
    _, _, y, _, uv = oracle.toggle_prior_predictive(m, np.zeros(19), n, seed=12, want_y=True, want_uv=True)
    assert np.all(uv == 1.0)
    y = y.ravel()
    sd = mu * sigma
    N = y.size
    assert abs(y.mean() - (1.0 + mu)) < Z * sd / np.sqrt(N), y.mean()
    assert abs(y.var() - sd ** 2) < Z * sd ** 2 * np.sqrt(2.0 / N), (y.var(), sd ** 2)


def test_v_represses_u():
    T, C = 200, 2000
    base = (300.0, 0.1, 0.1, 40.0, 0.0, 4.0, 0.0)
    low_v = fixed(base, T, C)                                # alpha_v = 0: v sits near the floor
    high_v = fixed(base[:4] + (40.0,) + base[5:], T, C)      # alpha_v = 40, beta_v = 0: v ~ 600
    _, _, y_lo, _ = oracle.toggle_prior_predictive(low_v, np.zeros(19), 1, seed=1, want_y=True)
    _, _, y_hi, _ = oracle.toggle_prior_predictive(high_v, np.zeros(19), 1, seed=1, want_y=True)
    # v ~ 1: u is driven by alpha_u / 2 (large); v large: p_u = v^4 kills production, u -> floor
    assert y_lo.mean() > 300.0 + 500.0
    assert y_hi.mean() < 300.0 + 10.0


def test_quantiles_distance_floor_and_prior():
    m = {"lo": PAPER_LO, "hi": PAPER_HI, "T": 120, "C": 1999}
    rng = np.random.default_rng(0)
    q_obs = np.sort(rng.uniform(100, 600, 19))
    theta, summ, y, dist = oracle.toggle_prior_predictive(m, q_obs, 12, seed=7, want_y=True)
    levels = np.arange(1, 20) / 20.0
    for i in range(12):
        np.testing.assert_allclose(summ[i], np.quantile(y[i], levels, method="linear"), rtol=1e-12)
    np.testing.assert_allclose(dist, np.linalg.norm(summ - q_obs, axis=1), rtol=1e-13)
    assert y.min() >= 1.0


def test_prior_is_the_paper_box():
    m = {"lo": PAPER_LO, "hi": PAPER_HI, "T": 2, "C": 1}
    theta, _, _, _ = oracle.toggle_prior_predictive(m, np.zeros(19), 20_000, seed=5)
    for j in range(7):
        lo, hi = PAPER_LO[j], PAPER_HI[j]
        assert stats.kstest(theta[:, j], "uniform", args=(lo, hi - lo)).pvalue > 1e-4
    c = np.corrcoef(theta.T)
    assert np.all(np.abs(c[np.triu_indices(7, 1)]) < Z / np.sqrt(theta.shape[0]))


def test_sharding_and_threads():
    m = {"lo": PAPER_LO, "hi": PAPER_HI, "T": 30, "C": 64}
    q = np.linspace(200, 500, 19)
    _, s_all, _, d_all = oracle.toggle_prior_predictive(m, q, 40, seed=2, n_threads=1)
    _, s_part, _, d_part = oracle.toggle_prior_predictive(m, q, 10, seed=2, base=25, n_threads=3)
    np.testing.assert_array_equal(d_all[25:35], d_part)
    np.testing.assert_array_equal(s_all[25:35], s_part)
    _, _, _, d_sub = oracle.toggle_prior_predictive(m, q, 40, seed=2, sub=1)
    assert not np.allclose(d_all, d_sub)
