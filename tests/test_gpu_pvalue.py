"""GPU parity of the prior-predictive p-value sweep (C ABI vs CPU oracle)."""
import numpy as np
import pytest
from scipy import stats

import oracle
from gpu_common import BAND, require_gpu, to_np, torch
from paper_1902_09046_gb300 import workloads

pytestmark = pytest.mark.gpu

# |dybar| <= lambda |dz_0| + mean |dz_t|, with |dz| <= 1e-6 for binary32 normals
def ybar_tol(lams):
    return 1e-6 * (1.0 + np.asarray(lams, dtype=np.float64))[:, None]


def run(binding, lams, n_obs, M, ybar_obs, seed):
    lt = torch.from_numpy(np.asarray(lams, dtype=np.float64)).cuda()
    out = binding.pvalue_sweep(lt, n_obs, M, ybar_obs, seed, want_ybar=True)
    torch.cuda.synchronize()
    return to_np(out["counts"]).astype(np.int64), to_np(out["p"]), to_np(out["ybar"])


@pytest.mark.parametrize("n_obs,M", [(50, 20_011), (1, 4097), (2, 300), (3, 1), (7, 999)])
def test_sweep_parity(n_obs, M):
    binding = require_gpu()
    lams = workloads.pvalue_lambdas()
    ybar_obs = workloads.pvalue_observed_ybar()
    c_g, p_g, y_g = run(binding, lams, n_obs, M, ybar_obs, seed=2)
    c_o, p_o, y_o = oracle.pvalue_sweep(lams, n_obs, M, ybar_obs, seed=2, want_ybar=True)
    err = np.abs(y_g - y_o)
    print(f"n={n_obs} M={M}: max |ybar err| {err.max():.3g}, max err/(1+lambda) "
          f"{(err / (1 + lams[:, None])).max():.3g}")
    assert np.all(err <= ybar_tol(lams))
    # the GPU count is exactly its own indicator sum
    np.testing.assert_array_equal(c_g, (np.abs(y_g) >= abs(ybar_obs)).sum(axis=1))
    # indicators agree with the oracle outside the band, which is set per
    # lambda from the stated ybar error: a data set can change side only if
    # | |ybar| - |ybar_obs| | is below the largest error the two sides can
    # have, so band_k = max(BAND |ybar_obs|, 2 ybar_tol(lambda_k))
    a = abs(ybar_obs)
    band_w = np.maximum(BAND * a, 2.0 * ybar_tol(lams))
    outside = np.abs(np.abs(y_o) - a) >= band_w
    np.testing.assert_array_equal((np.abs(y_g) >= a)[outside], (np.abs(y_o) >= a)[outside])
    band = (~outside).sum(axis=1)
    print(f"n={n_obs} M={M}: data sets inside the band per lambda {band.tolist()}")
    assert np.all(np.abs(c_g - c_o.astype(np.int64)) <= band)
    np.testing.assert_array_equal(p_g, c_g / M)


def test_full_sweep_matches_closed_form():
    binding = require_gpu()
    w = workloads.pvalue_sweep_workload()
    lt = torch.from_numpy(w.lambdas).cuda()
    out = binding.pvalue_sweep(lt, w.n_obs, w.m_sets, w.ybar_obs, w.seed, want_ybar=True)
    torch.cuda.synchronize()
    p = to_np(out["p"])
    s = np.sqrt(w.lambdas ** 2 + 1.0 / w.n_obs)
    ref = 2 * stats.norm.sf(abs(w.ybar_obs) / s)
    se = np.sqrt(np.maximum(ref * (1 - ref), 1e-12) / w.m_sets)
    assert np.all(np.abs(p - ref) < 4.5 * se + 1.0 / w.m_sets), np.max(np.abs(p - ref) / se)
    assert to_np(out["counts"])[0] == 0
    # the first 2000 data sets of every lambda, recomputed by the oracle
    _, _, y_o = oracle.pvalue_sweep(w.lambdas, w.n_obs, 2000, w.ybar_obs, w.seed, want_ybar=True)
    y_g = to_np(out["ybar"][:, :2000])
    assert np.all(np.abs(y_g - y_o) <= ybar_tol(w.lambdas))


def test_invalid_arguments():
    binding = require_gpu()
    lt = torch.ones(3, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PPABCError):
        binding.pvalue_sweep(lt, 0, 10, 1.0, 1)
    with pytest.raises(binding.PPABCError):
        binding.pvalue_sweep(lt, 10, 0, 1.0, 1)


# ---------------------------------------------------------------------------
# Weak-informativity test (Algorithm 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,n_obs", [(2000, 50), (4097, 7), (1, 3), (16384, 50)])
def test_weakinf_matches_oracle(N, n_obs):
    binding = require_gpu()
    lams = np.array([0.05, 0.5, 1.0, 2.0, 10.0, 100.0])
    lam0, alpha = 1.0, 0.05
    out = binding.weakinf_test(torch.from_numpy(lams).cuda(), lam0, n_obs, N, alpha, seed=9,
                               want_counts=True)
    torch.cuda.synchronize()
    g_o, c_o = oracle.weakinf(lams, lam0, n_obs, N, alpha, seed=9, want_counts=True)
    c_g = to_np(out["counts"]).astype(np.int64)
    diff = np.abs(c_g - c_o.astype(np.int64))
    # a count differs only where binary32 normals move |ybar| across a near-tie
    print(f"N={N}: counts equal for {np.mean(diff == 0):.6f} of base sets, max diff {diff.max()}")
    assert diff.max() <= 2
    assert np.mean(diff == 0) >= 0.999
    assert np.all(np.abs(to_np(out["gamma"]) - g_o) <= 2.0 / N)


def test_weakinf_invalid():
    binding = require_gpu()
    lt = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PPABCError):
        binding.weakinf_test(lt, 1.0, 50, binding.WEAKINF_MAX_SETS + 1, 0.05, 1)
    with pytest.raises(binding.PPABCError):
        binding.weakinf_test(lt, 1.0, 50, 100, 0.0, 1)
