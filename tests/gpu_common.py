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


def band_check(idx_gpu, idx_orc, d_orc, eps_orc, band=BAND):
    """Every index in exactly one of the two accept sets lies within the band
    around epsilon (computed from the oracle's distances); returns the number
    of band members that differ."""
    diff = np.setxor1d(np.asarray(idx_gpu, dtype=np.int64), np.asarray(idx_orc, dtype=np.int64))
    bad = [int(i) for i in diff if abs(d_orc[int(i)] - eps_orc) >= band * eps_orc]
    assert not bad, f"{len(bad)} accept decisions differ outside the band, e.g. {bad[:5]}"
    return diff.size
