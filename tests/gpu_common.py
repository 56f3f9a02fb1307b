"""Shared fixtures for the GPU parity tests (imported only by -m gpu tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_09046_gb300 import binding, build
    build.build()
    binding.device_check()
    return binding


def to_np(t):
    return t.detach().cpu().numpy()


# Tolerances and where they come from:
#  * a binary32 Box-Muller normal differs from the binary64 one by a few ulp
#    of the radius: |dz| <= 1e-6 (r <= 5.77, ~3 ulp);
#  * a binary32 prior draw is within 2 ulp: |dtheta| <= 5e-7 on |theta| <= 2;
#  * the compensated binary32 path keeps every summary within 2e-5 of the
#    binary64 path and the relative distance error below 1e-5 (measured
#    maxima are printed by the tests);
#  * accept sets must agree outside the band |d - eps| < 1e-6 eps.
Z_ATOL = 1e-6
THETA_ATOL = 5e-7
SUMM_ATOL = 2e-5
DIST_RTOL = 1e-5
BAND = 1e-6


def posterior_bounds(th_gpu, th_orc, idx):
    """Bounds on the posterior mean and variance differences over one index
    set when the two sides hold the same samples up to the per-element
    difference delta_i = theta_gpu,i - theta_orc,i (|delta_i| <= d).

    mean: |dm| <= max |delta_i| = d (a mean of the delta_i).
    var: with a_i = theta_i - m and e_i = delta_i - mean(delta), the centred
    sums differ by 2 sum a_i e_i + sum e_i^2 = 2 sum a_i delta_i + sum e_i^2
    (sum a_i = 0), so (k - 1) |dv| <= 2 d sum |a_i| + k d^2
    <= 2 d sqrt(k (k - 1) v) + k d^2 (Cauchy-Schwarz).
    A rounding allowance of 1e-12 relative is added to each (binary64 and
    double-float reductions).  Returns (mean_tol[3], var_tol[3], d[3])."""
    idx = np.asarray(idx, dtype=np.int64)
    k = idx.size
    a, b = th_gpu[idx].astype(np.float64), th_orc[idx].astype(np.float64)
    d = np.abs(a - b).max(axis=0)
    m = b.mean(axis=0)
    v = b.var(axis=0, ddof=1) if k > 1 else np.full(3, np.nan)
    mean_tol = d + 1e-12 * (np.abs(m) + 1e-300)
    var_tol = (2 * d * np.sqrt(k * (k - 1) * v) + k * d ** 2) / max(k - 1, 1) + 1e-12 * v
    return mean_tol, var_tol, d


def band_check(idx_gpu, idx_orc, d_orc, eps_orc, band=BAND):
    """Every index in exactly one of the two accept sets lies within the band
    around epsilon (computed from the oracle's distances); returns the number
    of band members that differ."""
    diff = np.setxor1d(np.asarray(idx_gpu, dtype=np.int64), np.asarray(idx_orc, dtype=np.int64))
    bad = [int(i) for i in diff if abs(d_orc[int(i)] - eps_orc) >= band * eps_orc]
    assert not bad, f"{len(bad)} accept decisions differ outside the band, e.g. {bad[:5]}"
    return diff.size
