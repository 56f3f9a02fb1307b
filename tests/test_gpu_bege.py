"""GPU parity of the BEGE log-likelihood (C ABI vs the binary64 CPU oracle).

Tolerance: the oracle forms F(u +- h) as two sums of 100 products of
incomplete gamma values and divides their difference by 2h (h = 1e-5).  Each
value carries the rounding of its exponent -x + a ln x - lnGamma(a): about
eps (x + a |ln x| + |lnGamma(a)|) relative, i.e. ~1e-15 for shapes near 1 and
~1e-13 for shapes in the hundreds, and the difference divides that by h.  The
GPU takes the difference node by node (no cancellation) and evaluates the
per-node work in double-float (48 bits): its own error, about 2^-48 times the
same exponent size, is far inside the oracle's.  So step t allows
  |d log f_t| <= 1e-13 (1 + s_t ln(2 + s_t)) / (h f_t),  s_t = p_{t-1} + n_{t-1},
with f_t from the oracle, and a particle the sum of that plus 1e-12 |ll|."""
import numpy as np
import pytest

import oracle
from gpu_common import require_gpu, to_np, torch
from paper_1902_09046_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H = W.BEGE_H


def _edge_particles():
    """Columns that end early: zero scale, negative scale, a shape driven
    below zero by phi_n+ < 0, and a tiny positive-shock scale whose grid
    cannot reach the returns (f = 0)."""
    ref = np.array(W.BEGE_THETA_REF)
    cols = []
    for k, v in ((1, 0.0), (6, -0.05)):
        c = ref.copy()
        c[k] = v
        cols.append(c)
    c = ref.copy()
    c[8], c[6], c[7], c[5] = -0.2, 0.005, 0.0, 0.05
    cols.append(c)
    c = ref.copy()
    c[1], c[0], c[6] = 1e-4, 1e-4, 1e-4
    cols.append(c)
    return np.stack(cols, axis=1)


def _shape_sums(theta, r):
    """p_{t-1} + n_{t-1} at every step (tolerance helper; NaN once invalid)."""
    n_p, T = theta.shape[1], len(r)
    out = np.full((n_p, T), np.nan)
    for i in range(n_p):
        p0, sp, rp, fpp, fpm, n0, sn, rn, fnp, fnm, mu = theta[:, i]
        p, n = p0, n0
        for t in range(T):
            if not (p > 0 and n > 0 and sp > 0 and sn > 0):
                break
            out[i, t] = p + n
            u = r[t] - mu
            p = p0 + rp * p + (fpp if u >= 0 else fpm) * u * u / (2 * sp * sp)
            n = n0 + rn * n + (fnp if u >= 0 else fnm) * u * u / (2 * sn * sn)
    return out


def _compare(theta, r, ll_gpu, logf_gpu, h=H):
    ll_o, dens = oracle.bege_loglik(theta, r, h, want_dens=True)
    fin_o, fin_g = np.isfinite(ll_o), np.isfinite(ll_gpu)
    s_t = _shape_sums(theta, r)
    with np.errstate(divide="ignore", invalid="ignore"):
        noise = 1e-13 * (1 + s_t * np.log(2 + s_t)) / h      # absolute rounding scale of f_t
        tol_t = np.where(dens > 0, noise / dens, 0.0)
    # A particle may end (-inf) on one side only where the deciding step's
    # density is within the rounding scale on the other side.
    for i in np.flatnonzero(fin_o != fin_g):
        if fin_o[i]:
            t0 = int(np.flatnonzero(logf_gpu[i] == -np.inf)[0])
            assert dens[i, t0] <= 2 * noise[i, t0], (i, t0, dens[i, t0], noise[i, t0])
        else:
            zero = np.flatnonzero(dens[i] <= 0)
            assert zero.size, f"particle {i}: the oracle ends it on a shape, the GPU does not"
            t0 = int(zero[0])
            assert np.exp(logf_gpu[i, t0]) <= 2 * noise[i, t0], (i, t0, logf_gpu[i, t0], noise[i, t0])
    both = fin_o & fin_g
    tol = np.nansum(tol_t, axis=1) + 1e-12 * np.abs(np.where(both, ll_o, 0.0))
    err = np.abs(ll_gpu - ll_o)
    assert np.all(err[both] <= tol[both]), (err[both].max(), tol[both][np.argmax(err[both])])
    live = (dens > 0) & np.isfinite(logf_gpu)
    e = np.abs(logf_gpu[live] - np.log(dens[live]))
    bad = np.flatnonzero(e > tol_t[live])
    if bad.size:
        w = bad[np.argsort(-(e[bad] / tol_t[live][bad]))[:5]]
        raise AssertionError("per-step log f outside tolerance: " + "; ".join(
            f"f={dens[live][k]:.4g} s={s_t[live][k]:.4g} err={e[k]:.3g} tol={tol_t[live][k]:.3g}" for k in w))
    worst = np.max(err[both] / np.maximum(tol[both], 1e-300)) if both.any() else 0.0
    return int(both.sum()), int((fin_o != fin_g).sum()), float(err[both].max() if both.any() else 0.0), float(worst)


def test_small_parity_prior_and_ref_particles():
    binding = require_gpu()
    r = W.bege_returns()[:120]
    theta = np.hstack([W.bege_particles(128, seed=6),
                       W.bege_particles(124, seed=8, centre=W.BEGE_THETA_REF, rel_spread=0.05),
                       _edge_particles()])
    out = binding.bege_loglik(torch.from_numpy(theta).cuda(), torch.from_numpy(r).cuda(), H, want_logf=True)
    ll, logf = to_np(out["ll"]), to_np(out["logf"])
    n_fin, n_edge, err, worst = _compare(theta, r, ll, logf)
    assert n_fin > 100 and n_edge <= 2
    assert np.all(~np.isfinite(ll[-4:]))
    print(f"BEGE T=120: {n_fin} finite on both sides of {theta.shape[1]}, {n_edge} ended on one side "
          f"at a rounding-level density, max |dll| {err:.3g}, worst err/tol {worst:.3f}")


@pytest.mark.parametrize("n_p,T", [(1, 1), (3, 2), (33, 7), (5, 257)])
def test_ragged_sizes(n_p, T):
    binding = require_gpu()
    r = W.bege_returns(T=T, seed=9)
    theta = W.bege_particles(n_p, seed=10, centre=W.BEGE_THETA_REF, rel_spread=0.03)
    out = binding.bege_loglik(torch.from_numpy(theta).cuda(), torch.from_numpy(r).cuda(), H, want_logf=True)
    _compare(theta, r, to_np(out["ll"]), to_np(out["logf"]))


def test_full_size_workload_sampled():
    """The benchmark's launch (1024 particles x 1099 months); the oracle
    checks a sample of particles over the whole series."""
    binding = require_gpu()
    r = W.bege_returns()
    theta = W.bege_particles(W.BEGE_N_PARTICLES, seed=6, centre=W.BEGE_THETA_REF, rel_spread=0.05)
    out = binding.bege_loglik(torch.from_numpy(theta).cuda(), torch.from_numpy(r).cuda(), H, want_logf=True)
    ll, logf = to_np(out["ll"]), to_np(out["logf"])
    pick = np.random.default_rng(12).choice(theta.shape[1], 12, replace=False)
    n_fin, n_edge, err, worst = _compare(theta[:, pick], r, ll[pick], logf[pick])
    print(f"BEGE T=1099 sample: {n_fin} finite of {len(pick)}, {n_edge} edge, max |dll| {err:.3g}, "
          f"worst err/tol {worst:.3f}")


def test_invalid_arguments():
    binding = require_gpu()
    lib = binding.load_library()
    th = torch.zeros((11, 4), dtype=torch.float64, device="cuda")
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    ll = torch.empty(4, dtype=torch.float64, device="cuda")
    ws_bytes = int(lib.bege_loglik_workspace_bytes(4, 8))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    P = binding._ptr
    assert lib.bege_loglik(P(th), 0, P(r), 8, H, P(ll), None, P(ws), ws_bytes, None) != 0
    assert lib.bege_loglik(P(th), 4, P(r), 0, H, P(ll), None, P(ws), ws_bytes, None) != 0
    assert lib.bege_loglik(P(th), 4, P(r), 8, 0.0, P(ll), None, P(ws), ws_bytes, None) != 0
    assert lib.bege_loglik(P(th), 4, P(r), 8, H, P(ll), None, P(ws), ws_bytes - 1, None) != 0
    assert lib.bege_loglik(None, 4, P(r), 8, H, P(ll), None, P(ws), ws_bytes, None) != 0
    assert lib.bege_loglik(P(th), 4, P(r), 8, H, P(ll), None, P(ws), ws_bytes, None) == 0


def test_extreme_regimes():
    """Columns that drive every branch of the per-node code: shapes in the
    hundreds (series past the reciprocal table, continued fraction past
    a + 66); a negative shape below 1 (singular density at the support edge);
    small sigma_n, whose delta = h / sigma_n is inside the Taylor bound at
    h = 1e-5 and above it at h = 1e-3 (every node takes both values)."""
    binding = require_gpu()
    ref = np.array(W.BEGE_THETA_REF)
    cols = []
    c = ref.copy(); c[0], c[2] = 8.0, 0.99; cols.append(c)                          # p up to ~400
    c = ref.copy(); c[5], c[7] = 5.0, 0.99; cols.append(c)                          # n up to ~250
    c = ref.copy(); c[0], c[2], c[5], c[7] = 8.0, 0.99, 5.0, 0.99; cols.append(c)   # both
    c = ref.copy(); c[5], c[7], c[8], c[9] = 0.05, 0.1, 1e-4, 1e-4; cols.append(c)   # n ~ 0.06
    # small sigma_n (delta 0.005 / 0.5 and 0.002 / 0.2) with a positive shock wide enough to cover the
    # returns (its support starts at -p sigma_p; the negative shock adds almost no left tail here)
    c = ref.copy(); c[0], c[1], c[6], c[8], c[9] = 2.0, 0.05, 2e-3, 1e-6, 1e-6; cols.append(c)
    c = ref.copy(); c[0], c[1], c[6], c[8], c[9] = 3.0, 0.06, 5e-3, 1e-6, 1e-6; cols.append(c)
    theta = np.stack(cols, axis=1)
    r = W.bege_returns(T=60, seed=13)
    for h in (H, 1e-3):
        out = binding.bege_loglik(torch.from_numpy(theta).cuda(), torch.from_numpy(r).cuda(), h, want_logf=True)
        n_fin, n_edge, err, worst = _compare(theta, r, to_np(out["ll"]), to_np(out["logf"]), h=h)
        assert n_fin == theta.shape[1], (h, n_fin)
        print(f"BEGE extreme regimes, h = {h:g}: {n_fin} finite of {theta.shape[1]}, {n_edge} edge, "
              f"max |dll| {err:.3g}, worst err/tol {worst:.3f}")
