"""GPU parity of the random number generation (C ABI vs CPU oracle)."""
import numpy as np
import pytest

import oracle
from gpu_common import Z_ATOL, require_gpu, to_np, torch

pytestmark = pytest.mark.gpu


def test_philox_words_bit_exact():
    binding = require_gpu()
    rng = np.random.default_rng(1)
    n = 100_003  # ragged
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0xFFFFFFFF, 0, 0xFFFFFFFF, 0]]
    for seed in (0, 1, 0xFFFFFFFF, 0xDEADBEEFCAFEF00D):
        got = to_np(binding.philox_raw(seed, torch.from_numpy(ctr).cuda()))
        np.testing.assert_array_equal(got, oracle.philox(seed, ctr))


def test_philox_empty_and_alignment():
    binding = require_gpu()
    empty = torch.empty((0, 4), dtype=torch.uint32, device="cuda")
    assert binding.philox_raw(5, empty).shape == (0, 4)


METHODS = [0, 1]  # binding.BM_POLY, binding.BM_TABLE


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("j0,n", [(0, 1), (0, 1_000_003), (7, 4097), (1 << 20, 999)])
def test_normals_match_oracle(j0, n, method):
    binding = require_gpu()
    for (c1, c2, tag) in ((0, 0, 1), (12345, 3, 1), (7, 0, 0)):
        z = to_np(binding.normals(99, c1, c2, tag, j0, n, method=method)).astype(np.float64)
        zo = oracle.stream_normals(99, c1, c2, tag, j0, n)
        err = np.abs(z - zo)
        assert err.max() <= Z_ATOL, err.max()
    print(f"max |z_gpu - z_oracle| = {err.max():.3g}")


def test_normal_moments_on_gpu():
    binding = require_gpu()
    z = binding.normals(2024, 5, 0, 1, 0, 1 << 24).double()
    n = z.numel()
    assert abs(z.mean().item()) < 4.5 / np.sqrt(n)
    assert abs(z.var().item() - 1) < 4.5 * np.sqrt(2.0 / n)


@pytest.mark.parametrize("method", METHODS)
def test_box_muller_exhaustive_over_both_uniforms(method):
    """Every one of the 2^23 uniforms, once as the radius word and once as the
    angle word, against the binary64 oracle transform on the same words, for
    both binary32 evaluations (polynomial and table-driven).
    Bound: |dz| <= 1.6e-7 r + 1e-9 (radius within ~1 ulp, sin/cos within ~1
    ulp absolute, product rounding)."""
    binding = require_gpu()
    m = np.arange(1 << 23, dtype=np.uint64)
    rng = np.random.default_rng(9)
    low = rng.integers(0, 512, size=m.size, dtype=np.uint64)   # the 9 bits the uniform drops
    words = ((m << np.uint64(9)) | low).astype(np.uint32)
    for fixed in (0x00000000, 0x40000000, 0x9E3779B9, 0xFFFFFFFF):
        for as_radius in (True, False):
            w = np.empty((words.size, 2), dtype=np.uint32)
            w[:, 0 if as_radius else 1] = words
            w[:, 1 if as_radius else 0] = fixed
            z = to_np(binding.box_muller(torch.from_numpy(w).cuda(), method=method)).astype(np.float64)
            zo = oracle.box_muller_words(w)
            r = np.hypot(zo[:, 0], zo[:, 1])
            err = np.abs(z - zo).max(axis=1)
            worst = np.max(err / (1.6e-7 * r + 1e-9))
            assert worst <= 1.0, (hex(fixed), as_radius, worst, err.max())
    print(f"Box-Muller exhaustive (method {method}): worst error / bound = {worst:.3f}")


@pytest.mark.parametrize("method", METHODS)
def test_packed_normals_bit_identical_to_scalar_transform(method):
    """The production kernels evaluate Box-Muller on packed binary32 pairs
    (the two pairs of a counter block side by side); the exhaustive test
    above checks the scalar transform.  Each packed component must be bit
    for bit the scalar result: the same operations in the same order, each
    rounded once."""
    binding = require_gpu()
    n_blocks = 1 << 20
    c1, c2, tag, seed = 4242, 7, 1, 31337
    ctr = np.zeros((n_blocks, 4), dtype=np.uint32)
    # counter of block b of stream (index c1, substream c2, tag): (tag, b, c2, c1)
    ctr[:, 1] = np.arange(n_blocks, dtype=np.uint32)
    ctr[:, 0], ctr[:, 2], ctr[:, 3] = tag, c2, c1
    words = binding.philox_raw(seed, torch.from_numpy(ctr).cuda())
    scalar = binding.box_muller(words.reshape(-1, 2).contiguous(), method=method).reshape(-1)
    packed = binding.normals(seed, c1, c2, tag, 0, 4 * n_blocks, method=method)
    np.testing.assert_array_equal(to_np(packed).view(np.uint32), to_np(scalar).view(np.uint32))
