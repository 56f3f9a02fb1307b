"""abc_select_static: the selection entry point for callers that cannot give
the library device memory (for example a service that forbids allocation once
it runs, or a plug-in that cannot reach its host framework's allocator).  Its
scratch is a static device array inside the library, shared by every call.

The GPU test calls it twice in a row through the C ABI, on different inputs
and in different modes, and checks each result against abc_select with a
caller-supplied workspace.  Selection is exact, so the comparison is exact;
the posterior moments use the 1e-12 relative tolerance of the other
selection tests.  This file is collected last so that a stop-at-first-failure
run has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1902_09046_gb300 import binding


def test_oversize_is_rejected_before_touching_the_gpu():
    lib = binding.load_library(build_if_missing=True)
    n = binding.STATIC_SELECT_MAX_N + 1
    rc = lib.abc_select_static(ctypes.c_void_p(256), n, 10, 0.0, None, 0, 0, 0, ctypes.c_void_p(256),
                               ctypes.c_void_p(256), ctypes.c_void_p(256), 10, ctypes.c_void_p(256),
                               None, None, None)
    assert rc == binding.PPABC_EINVAL
    assert b"at most" in lib.ppabc_last_error()


def _same(a, b):
    # only the first min(n_acc, cap) entries are written; the rest is untouched memory
    n = int(a["n_acc"].cpu()[0])
    assert n == int(b["n_acc"].cpu()[0])
    w = min(n, a["idx"].shape[0])
    np.testing.assert_array_equal(a["idx"][:w].cpu().numpy(), b["idx"][:w].cpu().numpy())
    np.testing.assert_array_equal(a["rec"][:w].cpu().numpy(), b["rec"][:w].cpu().numpy())
    assert a["eps"].cpu().numpy()[0] == b["eps"].cpu().numpy()[0]
    np.testing.assert_allclose(a["post"].cpu().numpy(), b["post"].cpu().numpy(), rtol=1e-12,
                               atol=1e-12, equal_nan=True)


@pytest.mark.gpu
def test_static_scratch_matches_workspace_version_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_09046_gb300 import build, workloads
    build.build()
    binding.device_check()

    # call 1: the 100 nearest of a 10^4-sample OU prior-predictive run, theta redrawn
    w = workloads.abc_small()
    sim = binding.abc_prior_predictive(w.model, w.y_obs, w.n_samples, w.seed, want_theta=False)
    s1 = binding.abc_select_static(sim["dist"], k=w.k_accept, model=w.model, seed=w.seed)
    r1 = binding.abc_select(sim["dist"], k=w.k_accept, model=w.model, seed=w.seed)
    torch.cuda.synchronize()
    _same(s1, r1)
    assert int(s1["n_acc"].cpu()[0]) == w.k_accept

    # call 2: threshold mode on a larger array with ties, theta given
    rng = np.random.default_rng(5)
    d = np.round(rng.gamma(2.0, 1.0, size=300_001), 2)
    dt = torch.from_numpy(d).cuda()
    th = torch.from_numpy(rng.normal(size=(3, d.size)).astype(np.float32)).cuda()
    eps = float(np.median(d))
    s2 = binding.abc_select_static(dt, k=0, eps=eps, theta=th)
    r2 = binding.abc_select(dt, k=0, eps=eps, theta=th)
    torch.cuda.synchronize()
    _same(s2, r2)
    assert int(s2["n_acc"].cpu()[0]) == int((d <= eps).sum())

    # a size the cluster selection serves (no scratch at all), theta given
    d4 = torch.from_numpy(d[:60_000].copy()).cuda()
    th4 = th[:, :60_000].contiguous()
    s4 = binding.abc_select_static(d4, k=600, theta=th4)
    r4 = binding.abc_select(d4, k=600, theta=th4)
    torch.cuda.synchronize()
    _same(s4, r4)
    assert int(s4["n_acc"].cpu()[0]) == 600

    # and once more in top-k mode on the second array (the scratch keeps state between calls)
    s3 = binding.abc_select_static(dt, k=777, theta=th)
    r3 = binding.abc_select(dt, k=777, theta=th)
    torch.cuda.synchronize()
    _same(s3, r3)
    assert math.isfinite(float(s3["eps"].cpu()[0]))
