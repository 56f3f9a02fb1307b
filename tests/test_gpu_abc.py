"""GPU parity of OU-ABC prior-predictive sampling and selection (C ABI vs the
CPU oracle), from small ragged cases up to the full 2^24 x 10^4 workload."""
import math

import numpy as np
import pytest

import oracle
from gpu_common import (BAND, DIST_RTOL, SUMM_ATOL, THETA_ATOL, band_check, posterior_bounds,
                        require_gpu, to_np, torch)
from paper_1902_09046_gb300 import workloads

pytestmark = pytest.mark.gpu


def check_posterior(post, th_g, th_o, idx_g, what):
    """Posterior mean and variance from the GPU (binary32 theta, redrawn from
    the prior counter) against the oracle's binary64 moments over the same
    index set, within the bound that the per-sample theta difference implies
    (posterior_bounds); prints the measured errors."""
    mean_o, var_o = oracle.moments(th_o, np.asarray(idx_g).astype(np.uint64))
    mean_tol, var_tol, d = posterior_bounds(th_g, th_o, idx_g)
    em, ev = np.abs(post[:3] - mean_o), np.abs(post[3:] - var_o)
    print(f"{what}: k={np.asarray(idx_g).size} max |dtheta| {d}; posterior mean abs err {em} "
          f"(bound {mean_tol}); var rel err {ev / var_o} (bound {var_tol / var_o})")
    assert np.all(em <= mean_tol), (em, mean_tol)
    assert np.all(ev <= var_tol), (ev, var_tol)
    return em, ev / var_o


def run_gpu(binding, model, y, n, seed, sub=0, base=0):
    out = binding.abc_prior_predictive(model, y, n, seed, substream=sub, sample_base=base,
                                       want_theta=True, want_summ=True)
    torch.cuda.synchronize()
    return to_np(out["theta"]).T.astype(np.float64), to_np(out["summ"]).T, to_np(out["dist"]), out


def compare_paths(model, y, n, seed, sub=0, base=0):
    binding = require_gpu()
    th_g, s_g, d_g, out = run_gpu(binding, model, y, n, seed, sub, base)
    th_o, s_o, d_o = oracle.ou_prior_predictive(model, y, n, seed=seed, sub=sub, base=base,
                                                want_summ=True)
    np.testing.assert_allclose(th_g, th_o, rtol=0, atol=THETA_ATOL)
    serr = np.abs(s_g - s_o).max()
    derr = (np.abs(d_g - d_o) / np.maximum(d_o, 1e-300)).max()
    print(f"n={n} S={model['n_steps']}: max |theta| err {np.abs(th_g - th_o).max():.3g}, "
          f"max |summary| err {serr:.3g}, max rel dist err {derr:.3g}")
    assert serr <= SUMM_ATOL
    assert derr <= DIST_RTOL
    return th_g, d_g, th_o, d_o, out


def test_small_workload_parity_and_accept_set():
    binding = require_gpu()
    w = workloads.abc_small()
    th_g, d_g, th_o, d_o, out = compare_paths(w.model, w.y_obs, w.n_samples, w.seed)
    sel = binding.abc_select(out["dist"], k=w.k_accept, model=w.model, seed=w.seed,
                             theta=out["theta"])
    sel_regen = binding.abc_select(out["dist"], k=w.k_accept, model=w.model, seed=w.seed)
    torch.cuda.synchronize()
    idx_g = to_np(sel["idx"]).astype(np.int64)
    idx_o = oracle.select_topk(d_o, w.k_accept).astype(np.int64)
    eps_o = np.sort(d_o)[w.k_accept - 1]
    ndiff = band_check(idx_g, idx_o, d_o, eps_o)
    print(f"accept-set differences inside the band: {ndiff}")
    assert int(to_np(sel["n_acc"])[0]) == w.k_accept
    assert np.all(np.diff(idx_g) > 0)
    # the GPU's own selection is exact on its own distances
    np.testing.assert_array_equal(idx_g, oracle.select_topk(d_g, w.k_accept).astype(np.int64))
    assert to_np(sel["eps"])[0] == np.sort(d_g)[w.k_accept - 1]
    rec = to_np(sel["rec"])
    np.testing.assert_array_equal(rec[:, :3], th_g[idx_g].astype(np.float32))
    np.testing.assert_array_equal(rec[:, 3], d_g[idx_g].astype(np.float32))
    # redrawing theta from the prior counter is bit-identical to the stored draw
    np.testing.assert_array_equal(to_np(sel_regen["rec"]), rec)
    np.testing.assert_array_equal(to_np(sel_regen["post"]), to_np(sel["post"]))
    # posterior moments vs the oracle's binary64 moments over the GPU's own
    # accepted set: the difference is bounded by the per-sample theta
    # difference alone, whatever the band members
    post = to_np(sel["post"])
    check_posterior(post, th_g, th_o, idx_g, "small workload")
    mean_oo, var_oo = oracle.moments(th_o, idx_o.astype(np.uint64))
    print(f"against the oracle's own accepted set: mean abs err {np.abs(post[:3] - mean_oo)}, "
          f"var rel err {np.abs(post[3:] - var_oo) / var_oo}")


# (steps, observations, samples, x0, horizon): th1 dt stays below 1 so the
# Euler-Maruyama recursion is stable for every prior draw.
@pytest.mark.parametrize("n_steps,n_obs,n,x0,t_end", [(37, 10, 5003, 0.0, 10.0),
                                                      (1000, 1, 1, 0.3, 10.0),
                                                      (4, 4, 129, -1.0, 0.4),
                                                      (250, 32, 1000, 2.0, 10.0),
                                                      (101, 7, 4099, 0.0, 10.0),
                                                      (40, 10, 100001, 0.0, 10.0)])
def test_ragged_models(n_steps, n_obs, n, x0, t_end):
    """n <= 98304 runs the pipelined kernel, n = 100001 the two-path kernel
    (with a ragged last CTA), both writing theta and the summaries."""
    model = workloads.ou_model(n_steps, t_end=t_end, n_obs=n_obs, x0=x0)
    y = np.linspace(-0.5, 1.0, n_obs)
    compare_paths(model, y, n, seed=11, sub=2)


def test_fixed_theta_and_sample_base_sharding():
    binding = require_gpu()
    model = {"lo": (1.2, 0.4, 0.5), "hi": (1.2, 0.4, 0.5), "x0": 0.0, "dt": 0.01, "n_steps": 500,
             "n_obs": 10}
    y = np.zeros(10)
    compare_paths(model, y, 3000, seed=5, base=123_456)
    w = workloads.abc_small()
    full = binding.abc_prior_predictive(w.model, w.y_obs, 8192, w.seed)
    half = binding.abc_prior_predictive(w.model, w.y_obs, 4096, w.seed, sample_base=4096)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(full["dist"])[4096:], to_np(half["dist"]))
    np.testing.assert_array_equal(to_np(full["theta"])[:, 4096:], to_np(half["theta"]))


@pytest.mark.parametrize("n", [1, 255, 256, 257, 100_001])
def test_theta_and_summary_outputs_leave_the_distances_unchanged(n):
    binding = require_gpu()
    w = workloads.abc_small()
    a = binding.abc_prior_predictive(w.model, w.y_obs, n, w.seed, sample_base=77, want_theta=False)
    b = binding.abc_prior_predictive(w.model, w.y_obs, n, w.seed, sample_base=77, want_theta=True)
    c = binding.abc_prior_predictive(w.model, w.y_obs, n, w.seed, sample_base=77, want_theta=True,
                                     want_summ=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(a["dist"]), to_np(b["dist"]))
    np.testing.assert_array_equal(to_np(a["dist"]), to_np(c["dist"]))
    np.testing.assert_array_equal(to_np(b["theta"]), to_np(c["theta"]))


@pytest.mark.parametrize("n_steps,n_obs,n", [(37, 10, 33), (1000, 1, 1), (4, 4, 129), (250, 32, 1000),
                                             (101, 7, 4099), (7, 7, 65), (9, 3, 31), (1000, 10, 98304),
                                             (1000, 10, 98305)])
def test_small_launch_pipeline_is_bit_identical(n_steps, n_obs, n):
    """Launches of up to 98304 samples run the warp-specialised pipeline
    (normals drawn by producer warps, paths walked by one warp), larger ones
    two interleaved paths per thread.  The same samples (same base) from a
    launch of each kind: distances, theta and summaries are equal bit for bit,
    for step counts that are not multiples of four and for several
    observations in one counter block."""
    binding = require_gpu()
    model = workloads.ou_model(n_steps, t_end=0.01 * n_steps, n_obs=n_obs)
    y = np.linspace(-0.5, 1.0, n_obs)
    big = max(n, 98305)
    for kw in ({"want_theta": False}, {"want_theta": True, "want_summ": True}):
        a = binding.abc_prior_predictive(model, y, n, 11, sample_base=5, **kw)
        b = binding.abc_prior_predictive(model, y, big, 11, sample_base=5, **kw)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_np(a["dist"]), to_np(b["dist"])[:n])
        if kw["want_theta"]:
            np.testing.assert_array_equal(to_np(a["theta"]), to_np(b["theta"])[:, :n])
            np.testing.assert_array_equal(to_np(a["summ"]), to_np(b["summ"])[:, :n])


def test_empty_and_invalid():
    binding = require_gpu()
    w = workloads.abc_small()
    out = binding.abc_prior_predictive(w.model, w.y_obs, 0, w.seed)
    assert out["dist"].numel() == 0
    with pytest.raises(binding.PPABCError):
        binding.abc_prior_predictive(dict(w.model, n_steps=5), w.y_obs, 10, w.seed)
    with pytest.raises(binding.PPABCError):
        binding.abc_prior_predictive(w.model, w.y_obs, 10, w.seed, sample_base=(1 << 32) - 5)
    d = torch.rand(10, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PPABCError):
        binding.abc_select(d, k=11, theta=torch.zeros((3, 10), device="cuda"))


# ---------------------------------------------------------------------------
# Selection on given distances: exact (bit-identical index sets)
# ---------------------------------------------------------------------------

def _select_cases():
    rng = np.random.default_rng(7)
    yield "ties", np.round(rng.gamma(2.0, 1.0, size=20_000), 1)
    d = rng.uniform(0, 1, size=100_003)
    d[::7] = d[3]
    yield "ragged_ties", d
    yield "one", np.array([0.5])
    yield "specials", np.array([np.nan, 0.0, -0.0, np.inf, 1.0, 0.0, np.nan, 2.0, np.inf, 1e-300])
    yield "large", rng.exponential(size=1 << 21)
    # small sizes with ties (one CTA)
    for n in (4095, 4096, 4097, 2049):
        yield f"edge{n}", np.round(rng.exponential(size=n), 2)
    # around the one-CTA selection's limit (12288 distances; 24576 where no
    # cluster fits) and the one-CTA slices of the cluster, heavy ties
    for n in (12288, 12289, 24575, 24576, 24577, 30001):
        yield f"mid{n}", np.round(rng.exponential(size=n), 1)
    # the cluster selection (24577 .. 196608 distances over eight CTAs): ties
    # spread over every slice, all keys equal, its largest size, and one more
    # (the multi-launch path)
    yield "cluster_ties150001", np.round(rng.exponential(size=150_001), 1)
    yield "cluster_equal50000", np.full(50_000, 0.25)
    yield "cluster_max196608", np.round(rng.exponential(size=196_608), 2)
    yield "over_cluster196609", rng.uniform(0, 1, size=196_609)
    # the multi-launch path with heavy ties across its 4096-distance tiles
    yield "tiles_ties300001", np.round(rng.exponential(size=300_001), 1)
    # distinct values: the radix passes stop once one key is left under the
    # prefix (after two or three passes here) ...
    for n in (1000, 24576, 30001):
        yield f"distinct{n}", rng.uniform(0, 1, size=n)
    # ... or only at the fifth (spacing 2^-43) or the last pass (2^-52), where
    # the values differ in their low bits
    for e in (43, 52):
        for n in (5000, 30001):
            yield f"lowbits{e}_{n}", 1.0 + rng.permutation(n) * 2.0 ** -e


@pytest.mark.parametrize("case", [c for c, _ in _select_cases()])
def test_select_exact_on_given_distances(case):
    binding = require_gpu()
    d = dict(_select_cases())[case]
    n = d.size
    theta = np.stack([np.arange(n, dtype=np.float32) * s for s in (1.0, -1.0, 0.5)])
    th_t = torch.from_numpy(theta).cuda()
    dt = torch.from_numpy(d).cuda()
    ks = sorted({1, min(n, 2), min(n, 5), n // 3 or 1, n})
    for k in ks:
        sel = binding.abc_select(dt, k=k, theta=th_t)
        torch.cuda.synchronize()
        idx_o = oracle.select_topk(d, k).astype(np.int64)
        np.testing.assert_array_equal(to_np(sel["idx"]).astype(np.int64), idx_o, err_msg=f"k={k}")
        assert int(to_np(sel["n_acc"])[0]) == k
        # epsilon is the k-th smallest distance (NaN above every number)
        acc = d[idx_o]
        eps_k = to_np(sel["eps"])[0]
        if np.isnan(acc).any():
            assert np.isnan(eps_k), f"k={k}"
        else:
            assert eps_k == acc.max(), f"k={k}"
        mean_o, var_o = oracle.moments(theta.T.astype(np.float64), idx_o.astype(np.uint64))
        post = to_np(sel["post"])
        np.testing.assert_allclose(post[:3], mean_o, rtol=1e-12, atol=1e-12)
        if k > 1:
            np.testing.assert_allclose(post[3:], var_o, rtol=1e-10)
        else:
            assert np.all(np.isnan(post[3:]))
    finite = d[np.isfinite(d)]
    for eps in (0.0, float(np.median(finite)) if finite.size else 0.0, math.inf, -1.0):
        sel = binding.abc_select(dt, k=0, eps=eps, theta=th_t)
        torch.cuda.synchronize()
        idx_o = oracle.select_eps(d, eps).astype(np.int64)
        n_acc = int(to_np(sel["n_acc"])[0])
        assert n_acc == idx_o.size
        np.testing.assert_array_equal(to_np(sel["idx"])[:n_acc].astype(np.int64), idx_o)
        assert to_np(sel["eps"])[0] == eps or (math.isinf(eps) and math.isinf(to_np(sel["eps"])[0]))


@pytest.mark.parametrize("n,k", [(65_536, 655), (150_001, 40_000)])
def test_cluster_selection_redraws_theta_bit_identically(n, k):
    """The cluster selection (24577 .. 196608 distances) with theta given and
    with theta redrawn from the prior counter: the same records and moments
    bit for bit, k accepted in index order, and the records' theta that of
    the accepted samples."""
    binding = require_gpu()
    w = workloads.abc_small()
    out = binding.abc_prior_predictive(w.model, w.y_obs, n, w.seed)
    sel = binding.abc_select(out["dist"], k=k, model=w.model, seed=w.seed, theta=out["theta"])
    sel_regen = binding.abc_select(out["dist"], k=k, model=w.model, seed=w.seed)
    torch.cuda.synchronize()
    d_g = to_np(out["dist"])
    idx_g = to_np(sel["idx"]).astype(np.int64)
    np.testing.assert_array_equal(idx_g, oracle.select_topk(d_g, k).astype(np.int64))
    np.testing.assert_array_equal(to_np(sel_regen["rec"]), to_np(sel["rec"]))
    np.testing.assert_array_equal(to_np(sel_regen["post"]), to_np(sel["post"]))
    th_g = to_np(out["theta"]).T
    np.testing.assert_array_equal(to_np(sel["rec"])[:, :3], th_g[idx_g])
    mean_o, var_o = oracle.moments(th_g.astype(np.float64), idx_g.astype(np.uint64))
    np.testing.assert_allclose(to_np(sel["post"])[:3], mean_o, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(to_np(sel["post"])[3:], var_o, rtol=1e-10)


def test_eps_infinity_accepts_every_sample():
    binding = require_gpu()
    w = workloads.abc_small()
    out = binding.abc_prior_predictive(w.model, w.y_obs, w.n_samples, w.seed)
    sel = binding.abc_select(out["dist"], k=0, eps=math.inf, theta=out["theta"])
    torch.cuda.synchronize()
    assert int(to_np(sel["n_acc"])[0]) == w.n_samples
    np.testing.assert_array_equal(to_np(sel["idx"]), np.arange(w.n_samples))
    th = to_np(out["theta"]).astype(np.float64)
    post = to_np(sel["post"])
    np.testing.assert_allclose(post[:3], th.mean(axis=1), rtol=1e-12)
    np.testing.assert_allclose(post[3:], th.var(axis=1, ddof=1), rtol=1e-10)


@pytest.mark.parametrize("n", [10_000, 60_000])
def test_cap_smaller_than_accepted_count(n):
    binding = require_gpu()
    d = torch.linspace(0, 1, n, dtype=torch.float64, device="cuda")
    th = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    sel = binding.abc_select(d, k=0, eps=0.5, theta=th, cap=100)
    torch.cuda.synchronize()
    assert int(to_np(sel["n_acc"])[0]) == int((to_np(d) <= 0.5).sum())
    np.testing.assert_array_equal(to_np(sel["idx"]), np.arange(100))


# ---------------------------------------------------------------------------
# Full-size workload: 2^24 samples x 10^4 steps, as the benchmark launches it
# ---------------------------------------------------------------------------

def test_large_workload_subset_parity_and_posterior_error():
    """First 2^16 samples of the 2^24 x 10^4 workload, accept 0.1%: accept set
    vs the oracle outside the band, posterior mean/var error stated."""
    binding = require_gpu()
    w = workloads.abc_large()
    n = 1 << 16
    k = int(0.001 * n)
    th_g, d_g, th_o, d_o, out = compare_paths(w.model, w.y_obs, n, w.seed)
    sel = binding.abc_select(out["dist"], k=k, model=w.model, seed=w.seed)
    torch.cuda.synchronize()
    idx_o = oracle.select_topk(d_o, k).astype(np.int64)
    eps_o = np.sort(d_o)[k - 1]
    idx_g = to_np(sel["idx"]).astype(np.int64)
    ndiff = band_check(idx_g, idx_o, d_o, eps_o)
    post = to_np(sel["post"])
    # precision study: the GPU's posterior moments (binary32 paths and theta,
    # binary64 or double-float reductions) against the binary64 oracle's over
    # the same accepted set, asserted within the theta-difference bound
    check_posterior(post, th_g, th_o, idx_g, f"2^16 subset of the 2^24 x 10^4 workload, band diffs {ndiff}")
    mean_oo, var_oo = oracle.moments(th_o, idx_o.astype(np.uint64))
    print(f"against the oracle's own accepted set: mean abs err {np.abs(post[:3] - mean_oo)}, "
          f"var rel err {np.abs(post[3:] - var_oo) / var_oo}")


def test_full_size_workload_sampled():
    binding = require_gpu()
    w = workloads.abc_large()
    N, k = w.n_samples, w.k_accept
    out = binding.abc_prior_predictive(w.model, w.y_obs, N, w.seed, want_theta=False)
    sel = binding.abc_select(out["dist"], k=k, model=w.model, seed=w.seed)
    torch.cuda.synchronize()
    d = out["dist"]
    eps = float(to_np(sel["eps"])[0])
    idx = sel["idx"].long()
    assert int(to_np(sel["n_acc"])[0]) == k
    # properties at any size: accepted are the k smallest
    assert float(d[idx].max()) == eps
    assert int((d < eps).sum()) <= k <= int((d <= eps).sum())
    # sampled outputs recomputed one by one by the oracle
    rng = np.random.default_rng(3)
    acc = to_np(idx)
    picks = np.concatenate([rng.choice(acc, 24, replace=False),
                            rng.integers(0, N, 24),
                            [0, N - 1]])
    d_host = to_np(d)
    for i in picks:
        th_o, _, d_o = oracle.ou_prior_predictive(w.model, w.y_obs, 1, seed=w.seed, base=int(i))
        assert abs(d_host[i] - d_o[0]) <= DIST_RTOL * d_o[0], (i, d_host[i], d_o[0])
    # every sampled accepted sample is within the oracle's epsilon band
    rec = to_np(sel["rec"])
    th1 = rec[:, 0]
    assert np.all((th1 >= 0.1) & (th1 <= 2.0))


# ---------------------------------------------------------------------------
# Algorithm 1 as stated: accept until M acceptances
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("chunk", [1000, 4096, 65_536])
def test_rejection_until_m_accepted(chunk):
    binding = require_gpu()
    w = workloads.abc_small()
    M = 200
    # epsilon at the 2% point of the oracle's distances: about 10^4 proposals needed
    _, _, d_o = oracle.ou_prior_predictive(w.model, w.y_obs, 30_000, seed=w.seed)
    eps = float(np.quantile(d_o, 0.02))
    res = binding.abc_rejection(w.model, w.y_obs, eps, M, 30_000, w.seed, chunk=chunk)
    torch.cuda.synchronize()
    assert res["n_acc"] == M
    idx = to_np(res["idx"]).astype(np.int64)
    assert np.all(np.diff(idx) > 0) and idx[-1] + 1 == res["tried"]
    # the oracle's first M acceptances in index order, up to band members
    acc_o = np.nonzero(d_o <= eps)[0]
    ref = acc_o[:M]
    diff = np.setxor1d(idx, ref)
    assert all(abs(d_o[i] - eps) < 1e-6 * eps for i in diff), diff
    assert abs(res["tried"] - (ref[-1] + 1)) <= (0 if diff.size == 0 else 30_000)
    rec = to_np(res["rec"])
    assert np.all(rec[:, 3] <= np.float32(eps) * (1 + 1e-6))


def test_rejection_budget_and_chunking_invariance():
    binding = require_gpu()
    w = workloads.abc_small()
    a = binding.abc_rejection(w.model, w.y_obs, 0.5, 10_000, 5_000, w.seed, chunk=777)
    b = binding.abc_rejection(w.model, w.y_obs, 0.5, 10_000, 5_000, w.seed, chunk=5_000)
    torch.cuda.synchronize()
    assert a["n_acc"] == b["n_acc"] < 10_000 and a["tried"] == b["tried"] == 5_000
    np.testing.assert_array_equal(to_np(a["idx"]), to_np(b["idx"]))
    np.testing.assert_array_equal(to_np(a["rec"]), to_np(b["rec"]))
    # the threshold form of abc_select on the same prefix gives the same set
    out = binding.abc_prior_predictive(w.model, w.y_obs, 5_000, w.seed, want_theta=False)
    sel = binding.abc_select(out["dist"], k=0, eps=0.5, model=w.model, seed=w.seed)
    torch.cuda.synchronize()
    n = int(to_np(sel["n_acc"])[0])
    np.testing.assert_array_equal(to_np(sel["idx"])[:n], to_np(a["idx"]))


# ---------------------------------------------------------------------------
# ABC recalibration
# ---------------------------------------------------------------------------

def test_recalibration_matches_oracle_on_the_same_pairs():
    """Same stored pairs on both sides (the GPU's own theta and summaries):
    neighbour sets, u and the recalibrated values are identical."""
    binding = require_gpu()
    w = workloads.abc_small()
    out = binding.abc_prior_predictive(w.model, w.y_obs, w.n_samples, w.seed, want_theta=True,
                                       want_summ=True)
    sel = binding.abc_select(out["dist"], k=w.k_accept, theta=out["theta"])
    for k in (1, 100, 731):
        rc = binding.abc_recalibrate(out["summ"], out["theta"], sel["idx"], k)
        torch.cuda.synchronize()
        u_o, rc_o = oracle.recalibrate(to_np(out["summ"]), to_np(out["theta"]), to_np(sel["idx"]), k)
        np.testing.assert_array_equal(to_np(rc["u"]), u_o)
        np.testing.assert_array_equal(to_np(rc["theta_rc"]), rc_o)
        if k == 1:
            assert np.all(to_np(rc["u"]) == 1.0)


def test_recalibration_identity_with_every_pair_accepted_and_a_neighbour():
    """q = n accepted and k = n neighbours: u = rank / n, so every value maps
    to itself (the rank ceil(u q) formed exactly, not from u q in binary64)."""
    binding = require_gpu()
    rng = np.random.default_rng(8)
    n = 300
    S = torch.from_numpy(rng.normal(size=(3, n))).cuda()
    th_np = rng.permutation(np.linspace(0.1, 0.9, 3 * n)).reshape(3, n).astype(np.float32)
    th = torch.from_numpy(th_np).cuda()
    acc = torch.arange(n, dtype=torch.int32, device="cuda").to(torch.uint32)
    rc = binding.abc_recalibrate(S, th, acc, n)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(rc["theta_rc"]), th_np)


def test_recalibration_end_to_end_against_oracle_pairs():
    """GPU pairs against the oracle's own pairs: u agrees to within the few
    neighbours that sit on the k-th distance band."""
    binding = require_gpu()
    w = workloads.abc_small()
    n, kacc, knn = 4000, 40, 200
    out = binding.abc_prior_predictive(w.model, w.y_obs, n, w.seed, want_theta=True, want_summ=True)
    sel = binding.abc_select(out["dist"], k=kacc, theta=out["theta"])
    rc = binding.abc_recalibrate(out["summ"], out["theta"], sel["idx"], knn)
    torch.cuda.synchronize()
    th_o, s_o, d_o = oracle.ou_prior_predictive(w.model, w.y_obs, n, w.seed, want_summ=True)
    acc = to_np(sel["idx"]).astype(np.uint32)
    u_o, _ = oracle.recalibrate(s_o.T.copy(), th_o.T.astype(np.float32).copy(), acc, knn)
    assert np.abs(to_np(rc["u"]) - u_o).max() <= 3.0 / knn


@pytest.mark.parametrize("n", [300, 24576, 24577])
def test_recalibration_ties_on_both_sides_of_the_shared_memory_limit(n):
    """Summaries on a coarse integer grid, so the k-th distance is shared by
    many pairs: the neighbour set must take the tied pairs in index order on
    the one-launch path (n up to 24576 keys in shared memory) and on the
    per-sample selection path above it; u and theta_rc identical to the
    oracle's."""
    binding = require_gpu()
    rng = np.random.default_rng(n)
    S_np = rng.integers(0, 4, size=(2, n)).astype(np.float64)
    th_np = rng.random(size=(3, n)).astype(np.float32)
    acc_np = rng.choice(n, size=7, replace=False).astype(np.uint32)
    S = torch.from_numpy(S_np).cuda()
    th = torch.from_numpy(th_np).cuda()
    acc = torch.from_numpy(acc_np.astype(np.int64)).cuda().to(torch.int32).to(torch.uint32)
    for k in (1, 37, n // 3, n - 1, n):
        rc = binding.abc_recalibrate(S, th, acc, k)
        torch.cuda.synchronize()
        u_o, rc_o = oracle.recalibrate(S_np, th_np, acc_np, k)
        np.testing.assert_array_equal(to_np(rc["u"]), u_o)
        np.testing.assert_array_equal(to_np(rc["theta_rc"]), rc_o)


# ---------------------------------------------------------------------------
# The exchange step of a sample-sharded job, on the device
# ---------------------------------------------------------------------------

def _sharded_select(binding, d, theta, k, cuts):
    """Per-shard abc_select + abc_select_candidates, concatenated in shard
    order (what the all-gather delivers), then abc_merge_candidates."""
    cands = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        kl = min(k, hi - lo)
        sel = binding.abc_select(d[lo:hi], k=kl, theta=theta[:, lo:hi].contiguous())
        cands.append(binding.abc_select_candidates(d[lo:hi], sel, kl, sample_base=lo))
    cat = {key: torch.cat([c[key] for c in cands], dim=-1) for key in ("dist", "index", "theta")}
    return binding.abc_merge_candidates(cat["dist"], cat["index"], cat["theta"].contiguous(), k)


@pytest.mark.parametrize("case", ["ou_small", "ties", "large"])
def test_sharded_merge_equals_unsharded(case):
    binding = require_gpu()
    rng = np.random.default_rng(21)
    if case == "ou_small":
        w = workloads.abc_small()
        out = binding.abc_prior_predictive(w.model, w.y_obs, w.n_samples, w.seed, want_theta=True)
        d, theta, k = out["dist"], out["theta"], w.k_accept
        cuts = [0, 3001, 3050, w.n_samples]          # uneven, one shard smaller than k
    elif case == "ties":
        n = 20_000
        d = torch.from_numpy(np.round(rng.exponential(size=n), 1)).cuda()   # heavy ties across shards
        theta = torch.from_numpy(rng.random((3, n)).astype(np.float32)).cuda()
        k, cuts = 777, [0, 5000, 12345, n]
    else:
        w = workloads.abc_large()
        n = 1 << 17
        out = binding.abc_prior_predictive(w.model, w.y_obs, n, w.seed, want_theta=True)
        d, theta, k = out["dist"], out["theta"], int(0.001 * n)
        cuts = [0, n // 2, n]
    ref = binding.abc_select(d, k=k, theta=theta)
    got = _sharded_select(binding, d, theta, k, cuts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(to_np(got["idx"]).astype(np.int64), to_np(ref["idx"]).astype(np.int64))
    np.testing.assert_array_equal(to_np(got["rec"]), to_np(ref["rec"]))
    assert int(to_np(got["n_acc"])[0]) == k
    assert to_np(got["eps"])[0] == to_np(ref["eps"])[0]
    # the same values in the same order; the grouping of the sums may differ
    np.testing.assert_allclose(to_np(got["post"]), to_np(ref["post"]), rtol=1e-12, atol=1e-15)
