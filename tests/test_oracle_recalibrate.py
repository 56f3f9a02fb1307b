"""Pins for the oracle's ABC recalibration (CPU only): a brute-force numpy
restatement of the definition on random inputs with ties, plus the identity
case where every pair is its own only neighbour (k = 1 gives u = 1)."""
import numpy as np

import oracle


def _numpy_recalibrate(S, th, acc, k):
    n = S.shape[1]
    q = acc.size
    u = np.zeros((3, q))
    for i, a in enumerate(acc):
        d = np.sqrt(((S - S[:, [a]]) ** 2).sum(axis=0))
        nn = np.lexsort((np.arange(n), d))[:k]
        for c in range(3):
            u[c, i] = np.count_nonzero(th[c, nn] <= th[c, a]) / k
    rc = np.zeros((3, q), dtype=np.float32)
    for c in range(3):
        srt = np.sort(th[c, acc])
        r = np.clip(np.ceil(u[c] * q).astype(np.int64), 1, q)
        rc[c] = srt[r - 1]
    return u, rc


def test_matches_numpy_definition():
    rng = np.random.default_rng(4)
    n, n_obs = 3000, 10
    # integer summaries: squared distances are exact in any summation order, so
    # the many ties are real ties and both sides break them by index
    S = rng.integers(-3, 4, size=(n_obs, n)).astype(np.float64)
    th = rng.uniform(0, 1, size=(3, n)).astype(np.float32)
    th[:, ::5] = th[:, 1:2]                            # and theta ties
    acc = np.sort(rng.choice(n, 60, replace=False)).astype(np.uint32)
    for k in (1, 7, 100, n):
        u, rc = oracle.recalibrate(S, th, acc, k)
        u_ref, rc_ref = _numpy_recalibrate(S, th, acc, k)
        np.testing.assert_allclose(u, u_ref, rtol=0, atol=0)
        np.testing.assert_array_equal(rc, rc_ref)
    u1, _ = oracle.recalibrate(S, th, acc, 1)
    assert np.all(u1 == 1.0)                           # the nearest pair is the pair itself
