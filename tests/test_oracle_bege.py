"""Pins of the oracle's BEGE log-likelihood (Sec. 4.2) to facts other than
its own code: scipy's incomplete gamma and closed forms, the limits of the
discretised distribution function, a Monte Carlo estimate of the integral
it discretises, the analytic derivative of that sum, and shape recursions
with closed-form solutions."""
import numpy as np
import pytest
from scipy import special, stats

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_incomplete_gamma_against_scipy_and_closed_forms():
    a = np.array([1e-3, 0.05, 0.3, 0.5, 1.0, 2.5, 10.0, 60.0, 300.0, 3e4])
    x = np.array([1e-10, 1e-4, 0.02, 0.5, 1.0, 2.9, 3.1, 11.0, 80.0, 290.0, 310.0, 1500.0, 3e4])
    A, X = np.meshgrid(a, x)
    P = oracle.gammainc_p(A, X)
    ref = special.gammainc(A, X)
    # Both evaluate exp(-x + a ln x - lnGamma(a)) times a series or fraction;
    # rounding the exponent's terms costs eps (x + a |ln x| + |lnGamma(a)|)
    # relative, which dominates for large a and x.
    scale = X + A * np.abs(np.log(X)) + np.abs(special.gammaln(A))
    assert np.all(np.abs(P - ref) <= 8 * np.finfo(float).eps * scale * ref + 1e-15)
    # a = 1: 1 - e^-x;  a = 1/2: erf(sqrt x);  a = 3: 1 - e^-x (1 + x + x^2/2).
    xs = np.array([1e-6, 0.1, 0.9, 2.0, 7.5, 40.0])
    np.testing.assert_allclose(oracle.gammainc_p(1.0, xs), -np.expm1(-xs), rtol=1e-13)
    np.testing.assert_allclose(oracle.gammainc_p(0.5, xs), special.erf(np.sqrt(xs)), rtol=1e-13)
    np.testing.assert_allclose(oracle.gammainc_p(3.0, xs), 1 - np.exp(-xs) * (1 + xs + xs ** 2 / 2),
                               rtol=1e-12, atol=1e-15)
    assert oracle.gammainc_p(2.0, 0.0) == 0.0 and oracle.gammainc_p(2.0, -1.0) == 0.0


def _grid(sp, p):
    w0 = 1e-4 - p * sp
    dw = (10 * sp * np.sqrt(p) - w0) / (oracle.BEGE_NW - 1)
    return w0 + np.arange(oracle.BEGE_NW + 1) * dw


@pytest.mark.parametrize("sp,sn,p,n", [(0.03, 0.05, 0.3, 0.8), (0.05, 0.02, 2.0, 0.4), (0.01, 0.04, 7.0, 3.0)])
def test_cdf_limits_are_the_grid_mass(sp, sn, p, n):
    """u -> +inf: every [1 - P(n, .)] is 1, so F is the p-mass on the grid,
    P(p, x_N) - P(p, x_0); u -> -inf: F -> 0; F is non-decreasing."""
    w = _grid(sp, p)
    mass = special.gammainc(p, (w[-1] + p * sp) / sp) - special.gammainc(p, (w[0] + p * sp) / sp)
    assert abs(oracle.bege_cdf(50.0, sp, sn, p, n) - mass) < 1e-13
    assert oracle.bege_cdf(-50.0, sp, sn, p, n) < 1e-12
    u = np.linspace(-0.5, 0.5, 401)
    F = oracle.bege_cdf(u, sp, sn, p, n)
    assert np.all(np.diff(F) >= -1e-15)


@pytest.mark.parametrize("sp,sn,p,n", [(0.03, 0.05, 0.3, 0.8), (0.05, 0.02, 2.0, 0.4)])
def test_cdf_against_monte_carlo_of_the_discretised_integral(sp, sn, p, n):
    """The sum is a left Riemann-Stieltjes sum of the monotone integrand
    1 - F_n(w - u) against F_p over the grid, so it lies within max_j dF_j
    of the integral over [w_0, w_N], which Monte Carlo estimates from gamma
    draws."""
    rng = np.random.default_rng(11)
    M = 2_000_000
    wp = sp * (rng.gamma(p, 1.0, M) - p)
    wn = sn * (rng.gamma(n, 1.0, M) - n)
    w = _grid(sp, p)
    inside = (wp >= w[0]) & (wp <= w[-1])
    dF = np.diff(special.gammainc(p, (w + p * sp) / sp))
    for q in (-0.08, -0.03, 0.0, 0.02, 0.06):
        est = np.mean(inside & (wp - wn <= q))
        se = np.sqrt(est * (1 - est) / M)
        F = oracle.bege_cdf(q, sp, sn, p, n)
        assert abs(F - est) <= dF.max() + 5 * se, (q, F, est)


@pytest.mark.parametrize("sp,sn,p,n", [(0.03, 0.05, 0.3, 2.5), (0.02, 0.03, 1.7, 2.2)])
def test_density_is_the_derivative_of_the_discretised_cdf(sp, sn, p, n):
    """d/du [1 - P(n, (w - u + n sn)/sn)] = g_n(w - u), the centred-gamma
    density, so the central difference must match sum_j g_n(w_{j-1} - u) dF_j
    up to O(h^2).  (n > 1 keeps g_n smooth; for n < 1 it is singular at the
    edge of its support and the difference quotient is not O(h^2) there.)"""
    h = 1e-5
    w = _grid(sp, p)
    dF = np.diff(special.gammainc(p, (w + p * sp) / sp))
    for u in (-0.1, -0.02, 0.0, 0.015, 0.05):
        g = stats.gamma.pdf((w[:-1] - u + n * sn) / sn, n) / sn
        exact = np.sum(g * dF)
        f = oracle.bege_density(u, sp, sn, p, n, h)
        assert abs(f - exact) <= 1e-6 * exact + 1e-7, (u, f, exact)


def _theta(p0=0.3, sp=0.03, rp=0.5, fpp=0.2, fpm=0.3, n0=0.6, sn=0.04, rn=0.4, fnp=0.05, fnm=0.4, mu=0.01):
    return np.array([[p0], [sp], [rp], [fpp], [fpm], [n0], [sn], [rn], [fnp], [fnm], [mu]])


def test_shape_recursion_closed_form_at_zero_innovations():
    """r_t = mu gives u_t = 0, so p_t = p0 (1 - rho^{t+1}) / (1 - rho): the
    log-likelihood is the sum of log f(0) at those shapes."""
    th = _theta()
    T, h = 12, 1e-5
    r = np.full(T, th[10, 0])
    ll, dens = oracle.bege_loglik(th, r, h, want_dens=True)
    p0, sp, rp, n0, sn, rn = th[0, 0], th[1, 0], th[2, 0], th[5, 0], th[6, 0], th[7, 0]
    want = 0.0
    for t in range(T):
        p = p0 * (1 - rp ** (t + 1)) / (1 - rp)
        n = n0 * (1 - rn ** (t + 1)) / (1 - rn)
        f = oracle.bege_density(0.0, sp, sn, p, n, h)
        # The closed form and the recursion round the shape differently (an
        # ulp), which the central difference turns into ~1e-11 of f.
        assert abs(dens[0, t] - f) <= 1e-9 * f
        want += np.log(f)
    assert abs(ll[0] - want) <= 1e-9 * T


def test_shape_recursion_branch_and_scale_without_memory():
    """With rho = 0 the shape at step t depends on u_{t-1} alone:
    p = p0 + phi_p^{sign} u^2 / (2 sp^2) and n = n0 + phi_n^{sign} u^2 / (2 sn^2),
    the sign picking phi^+ for u >= 0 and phi^- for u < 0."""
    th = _theta(rp=0.0, rn=0.0, fpp=0.05, fpm=0.35, fnp=0.01, fnm=0.5)
    mu = th[10, 0]
    u = np.array([0.04, -0.05, 0.02, -0.01, 0.0])
    h = 1e-5
    ll, dens = oracle.bege_loglik(th, u + mu, h, want_dens=True)
    p0, sp, fpp, fpm = th[0, 0], th[1, 0], th[3, 0], th[4, 0]
    n0, sn, fnp, fnm = th[5, 0], th[6, 0], th[8, 0], th[9, 0]
    for t in range(1, len(u)):
        up = u[t - 1]
        p = p0 + (fpp if up >= 0 else fpm) * up ** 2 / (2 * sp ** 2)
        n = n0 + (fnp if up >= 0 else fnm) * up ** 2 / (2 * sn ** 2)
        f = oracle.bege_density(u[t], sp, sn, p, n, h)
        assert abs(dens[0, t] - f) <= 1e-9 * f, t


def test_invalid_particles_are_minus_infinity():
    r = np.array([0.01, 0.05, 0.02, -0.01])
    th = np.hstack([_theta(), _theta(sp=0.0), _theta(sn=-0.1),
                    _theta(fnp=-0.2, sn=0.01, rn=0.0, n0=0.05)])  # n_1 < 0 after u_1 = 0.04 >= 0
    ll = oracle.bege_loglik(th, r, 1e-5)
    assert np.isfinite(ll[0])
    assert np.all(ll[1:] == -np.inf)
    # A return beyond the grid's reach (w_N = 10 sp sqrt(p) ~ 0.16 here): the
    # discretised distribution function is flat there, f = 0.
    ll, dens = oracle.bege_loglik(_theta(), np.array([0.01, 0.3]), 1e-5, want_dens=True)
    assert ll[0] == -np.inf and dens[0, 1] == 0.0 and dens[0, 0] > 0


def test_shape_overflow_is_minus_infinity_and_ends_quickly():
    """rho > 1 makes the shapes grow without bound; once one is not a finite
    number the particle ends (-inf) instead of summing a series of zero terms."""
    import time
    th = _theta(rp=8.0, rn=8.0)
    t0 = time.perf_counter()
    ll = oracle.bege_loglik(th, np.full(400, 0.01), 1e-5)
    assert ll[0] == -np.inf
    assert time.perf_counter() - t0 < 20.0
