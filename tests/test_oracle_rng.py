"""Pins for the oracle's random number generation (CPU only).

* Philox4x32-10 words are checked against an independent library
  implementation (Triton's ``tl.philox`` run by its CPU interpreter), on
  counters that exercise every lane and the 32-bit wrap.
* Uniforms and Box-Muller normals are checked against the distributions they
  must follow (moments within Monte Carlo error, Kolmogorov-Smirnov, lack of
  correlation), not against a retyped formula.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

import oracle

_TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def _k(out, seed, c0p, c1p, c2p, c3p, n: tl.constexpr):
        o = tl.arange(0, n)
        a, b, c, d = tl.philox(seed, tl.load(c0p + o), tl.load(c1p + o),
                               tl.load(c2p + o), tl.load(c3p + o))
        tl.store(out + o * 4 + 0, a)
        tl.store(out + o * 4 + 1, b)
        tl.store(out + o * 4 + 2, c)
        tl.store(out + o * 4 + 3, d)

    data = np.load(sys.argv[1])
    ctr, seeds = data["ctr"], data["seeds"]
    n = ctr.shape[0]
    res = []
    for s in seeds:
        cols = [torch.from_numpy(ctr[:, j].astype(np.int64)).to(torch.int32).view(torch.uint32)
                for j in range(4)]
        out = torch.zeros(n * 4, dtype=torch.int32).view(torch.uint32)
        _k[(1,)](out, int(s), cols[0], cols[1], cols[2], cols[3], n=n)
        res.append(out.view(torch.int32).numpy().astype(np.uint32).reshape(n, 4))
    np.save(sys.argv[2], np.stack(res))
""")


def test_philox_matches_triton_library(tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(12345)
    n = 64
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [1, 0, 0, 0]
    ctr[3] = [0, 1, 0, 0]
    ctr[4] = [0, 0, 1, 0]
    ctr[5] = [0, 0, 0, 1]
    seeds = np.array([0, 1, 2, 0xFFFFFFFF, 0x100000000, 0xDEADBEEFCAFEF00D], dtype=np.uint64)
    inp = tmp_path / "in.npz"
    outp = tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, seeds=seeds)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1")
    subprocess.run([sys.executable, str(script), str(inp), str(outp)], check=True, env=env,
                   timeout=600)
    ref = np.load(outp)
    for si, s in enumerate(seeds):
        got = oracle.philox(int(s), ctr)
        np.testing.assert_array_equal(got, ref[si], err_msg=f"seed {int(s):#x}")


def test_philox_key_and_counter_all_matter():
    base = np.array([[7, 11, 13, 17]], dtype=np.uint32)
    w0 = oracle.philox(5, base)
    assert not np.array_equal(w0, oracle.philox(6, base))
    assert not np.array_equal(w0, oracle.philox(5 + (1 << 32), base))
    for lane in range(4):
        c = base.copy()
        c[0, lane] ^= 1
        assert not np.array_equal(w0, oracle.philox(5, c))


def _words(n_blocks, seed=99):
    ctr = np.zeros((n_blocks, 4), dtype=np.uint32)
    # blocks 0..n_blocks-1 of the stream (index 0, substream 0, tag PATH)
    ctr[:, 1] = np.arange(n_blocks, dtype=np.uint32)
    ctr[:, 0] = 1
    return oracle.philox(seed, ctr).reshape(-1)


def test_words_are_uniform_bits():
    w = _words(1 << 18)
    # each of the 32 bits is set half of the time (4.5 standard errors)
    n = w.size
    for b in range(32):
        frac = ((w >> b) & 1).mean()
        assert abs(frac - 0.5) < 4.5 * 0.5 / np.sqrt(n), b
    # chi-square on the top 10 bits
    counts = np.bincount((w >> 22).astype(np.int64), minlength=1024)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4


def test_uniform_range_and_monotone():
    ws = [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF]
    us = [oracle.u01(w) for w in ws]
    assert all(0.0 < u < 1.0 for u in us)
    assert us == sorted(us)
    assert oracle.u01(0) == oracle.u01(511)          # 2^23 cells of 512 words
    assert oracle.u01(512) > oracle.u01(511)
    # cell midpoints are symmetric about 1/2
    assert oracle.u01(0) + oracle.u01(0xFFFFFFFF) == 1.0
    # the uniforms of many words pass a KS test against U(0,1)
    w = _words(1 << 16, seed=3)
    u = np.array([oracle.u01(int(x)) for x in w[:20000]])
    assert stats.kstest(u, "uniform").pvalue > 1e-4


@pytest.fixture(scope="module")
def normals():
    return oracle.stream_normals(seed=2024, c1=5, c2=0, tag=oracle.TAG_PATH, j0=0, n=2_000_000)


def test_normal_moments(normals):
    z = normals
    n = z.size
    assert abs(z.mean()) < 4.5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 4.5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 4.5 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(z)) < 4.5 * np.sqrt(24.0 / n)
    # the 23-bit uniforms bound |z| by sqrt(2 * 24 ln 2) ~ 5.77
    assert np.abs(z).max() <= np.sqrt(2 * 24 * np.log(2)) + 1e-12


def test_normal_ks_and_independence(normals):
    z = normals
    assert stats.kstest(z[:500_000], "norm").pvalue > 1e-4
    n = z.size
    # even/odd members of a Box-Muller pair, and successive normals, are uncorrelated
    for a, b in ((z[0::2], z[1::2]), (z[:-1], z[1:]), (z[:-4], z[4:])):
        r = np.corrcoef(a, b)[0, 1]
        assert abs(r) < 4.5 / np.sqrt(a.size), r
    # squared radius of a pair is chi-square with 2 degrees of freedom
    r2 = z[0::2] ** 2 + z[1::2] ** 2
    assert stats.kstest(r2[:500_000], "chi2", args=(2,)).pvalue > 1e-4


def test_stream_offsets_are_consistent():
    a = oracle.stream_normals(7, 3, 1, oracle.TAG_PATH, 0, 64)
    b = oracle.stream_normals(7, 3, 1, oracle.TAG_PATH, 13, 20)
    np.testing.assert_array_equal(a[13:33], b)
    c = oracle.stream_normals(7, 4, 1, oracle.TAG_PATH, 0, 64)
    d = oracle.stream_normals(7, 3, 2, oracle.TAG_PATH, 0, 64)
    e = oracle.stream_normals(7, 3, 1, oracle.TAG_PRIOR, 0, 64)
    for other in (c, d, e):
        assert not np.allclose(a, other)
