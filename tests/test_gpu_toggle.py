"""GPU parity of the toggle-switch prior predictive against the FP64 oracle.

The state is binary32 on the GPU and binary64 in the oracle.  With the 0.97
contraction per step the rounding differences stay at a few ulp of u and v
(measured cell errors are a few 1e-6 relative at most); the paper's model is
bistable, though, so a cell on the switching boundary could land in the other
state under rounding.  Parity is therefore stated per cell (at least 99.9% of
cells within rtol 1e-4) and, for the summaries, as rtol 1e-4 on every
quantile and on rho.
"""
import numpy as np
import pytest

import oracle
from gpu_common import require_gpu, to_np, torch
from paper_1902_09046_gb300 import workloads

pytestmark = pytest.mark.gpu


def _compare(model, n, seed, base=0, sub=0):
    binding = require_gpu()
    q = workloads.toggle_observed_quantiles()
    out = binding.toggle_prior_predictive(model, q, n, seed, substream=sub, sample_base=base,
                                          want_theta=True, want_summ=True, want_y=True)
    torch.cuda.synchronize()
    th_o, s_o, y_o, d_o = oracle.toggle_prior_predictive(model, q, n, seed, sub=sub, base=base,
                                                         want_y=True)
    th_g = to_np(out["theta"]).T.astype(np.float64)
    y_g = to_np(out["y"]).astype(np.float64)
    s_g = to_np(out["summ"]).T
    d_g = to_np(out["dist"])
    np.testing.assert_allclose(th_g, th_o, rtol=2.5e-7, atol=1e-6)
    rel = np.abs(y_g - y_o) / y_o
    frac_close = np.mean(rel <= 1e-4)
    q_rel = np.abs(s_g - s_o) / np.abs(s_o)
    d_rel = np.abs(d_g - d_o) / d_o
    print(f"T={model['T']} C={model['C']} n={n}: cells within 1e-4: {frac_close:.6f}, "
          f"max cell rel {rel.max():.3g}, median {np.median(rel):.3g}; "
          f"max quantile rel {q_rel.max():.3g}; max dist rel {d_rel.max():.3g}")
    return frac_close, rel, q_rel, d_rel


def test_small_toggle_parity():
    frac, rel, q_rel, d_rel = _compare(workloads.toggle_model(T=120, C=2000), 24, seed=3)
    assert frac >= 0.999
    assert np.median(rel) <= 1e-6
    assert q_rel.max() <= 1e-4
    assert d_rel.max() <= 1e-4


@pytest.mark.parametrize("T,C", [(2, 1), (3, 7), (600, 33), (101, 4097)])
def test_toggle_edge_sizes(T, C):
    frac, rel, q_rel, d_rel = _compare(workloads.toggle_model(T=T, C=C), 5, seed=9, base=1000, sub=2)
    assert frac >= 0.999
    assert q_rel.max() <= 1e-4
    assert d_rel.max() <= 1e-4


def test_paper_workload_sampled():
    """N = 8064 samples, T = 600, C = 8000 (the paper's benchmark size); a
    spread of samples recomputed by the oracle."""
    binding = require_gpu()
    model = workloads.toggle_model()
    q = workloads.toggle_observed_quantiles()
    N = 8064
    out = binding.toggle_prior_predictive(model, q, N, 1, want_summ=True)
    torch.cuda.synchronize()
    d = to_np(out["dist"])
    s = to_np(out["summ"])
    assert np.all(np.isfinite(d)) and np.all(d > 0)
    for i in (0, 1, 4031, 8063):
        _, s_o, _, d_o = oracle.toggle_prior_predictive(model, q, 1, 1, base=i)
        q_rel = np.abs(s[:, i] - s_o[0]) / s_o[0]
        assert q_rel.max() <= 1e-4, (i, q_rel.max())
        assert abs(d[i] - d_o[0]) / d_o[0] <= 1e-4
