"""Pins for the oracle's ABC recalibration (CPU only): a brute-force numpy
restatement of the definition on random inputs with ties, plus the identity
case where every pair is its own only neighbour (k = 1 gives u = 1)."""
import numpy as np

import oracle


def _numpy_recalibrate(S, th, acc, k):
    n = S.shape[1]
    q = acc.size
    u = np.zeros((3, q))
    cnt = np.zeros((3, q), dtype=np.int64)
    for i, a in enumerate(acc):
        d = np.sqrt(((S - S[:, [a]]) ** 2).sum(axis=0))
        nn = np.lexsort((np.arange(n), d))[:k]
        for c in range(3):
            cnt[c, i] = np.count_nonzero(th[c, nn] <= th[c, a])
            u[c, i] = cnt[c, i] / k
    rc = np.zeros((3, q), dtype=np.float32)
    for c in range(3):
        srt = np.sort(th[c, acc])
        r = np.clip((cnt[c] * q + k - 1) // k, 1, q)      # ceil(u q) with u = cnt / k, exactly
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


def test_all_pairs_as_neighbours_give_the_empirical_cdf():
    """k = n: every stored pair is a neighbour whatever the summaries, so u is
    the empirical distribution function of theta at theta_a, rank / n."""
    rng = np.random.default_rng(7)
    n = 500
    S = rng.normal(size=(4, n))
    th = rng.uniform(size=(3, n)).astype(np.float32)
    acc = np.arange(0, n, 3, dtype=np.uint32)
    u, _ = oracle.recalibrate(S, th, acc, n)
    for c in range(3):
        ranks = np.searchsorted(np.sort(th[c]), th[c, acc], side="right")
        np.testing.assert_array_equal(u[c], ranks / n)


def test_identity_when_every_pair_is_accepted_and_every_pair_is_a_neighbour():
    """With q = n and k = n, u = rank / n, so the ceil(u q)-th smallest
    accepted value is theta_a itself (distinct values)."""
    rng = np.random.default_rng(8)
    n = 300
    S = rng.normal(size=(3, n))
    th = rng.permutation(np.linspace(0.1, 0.9, 3 * n)).reshape(3, n).astype(np.float32)
    acc = np.arange(n, dtype=np.uint32)
    _, rc = oracle.recalibrate(S, th, acc, n)
    np.testing.assert_array_equal(rc, th)


def test_invariant_under_relabelling_and_monotone_maps():
    rng = np.random.default_rng(9)
    n, k = 800, 25
    S = rng.normal(size=(5, n))          # continuous: no distance ties
    th = rng.uniform(size=(3, n)).astype(np.float32)
    acc = np.sort(rng.choice(n, 40, replace=False)).astype(np.uint32)
    u, rc = oracle.recalibrate(S, th, acc, k)
    perm = rng.permutation(n)
    inv = np.argsort(perm)
    u2, rc2 = oracle.recalibrate(S[:, perm], th[:, perm], inv[acc].astype(np.uint32), k)
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(rc2, rc)
    # theta -> 2 theta + 1 is increasing and exact in binary32 here: u unchanged,
    # recalibrated values mapped the same way
    u3, rc3 = oracle.recalibrate(S, (2 * th + 1).astype(np.float32), acc, k)
    np.testing.assert_array_equal(u3, u)
    np.testing.assert_array_equal(rc3, (2 * rc + 1).astype(np.float32))


def test_small_case_worked_by_hand():
    """Summaries 0, 1, 3, 7 on a line, theta_1 = 0.1, 0.4, 0.2, 0.3.  For the
    pair at S = 1 the two nearest pairs are itself (d = 0) and S = 0 (d = 1),
    with theta 0.4 and 0.1: u = 2/2.  For S = 3 they are itself and S = 1
    (d = 2 beats d = 4): theta 0.2 and 0.4, u = 1/2.  Accepting both pairs
    (q = 2, sorted accepted theta 0.2, 0.4), u = 1 maps to the 2nd value, 0.4,
    and u = 1/2 to the 1st, 0.2."""
    S = np.array([[0.0, 1.0, 3.0, 7.0]])
    th = np.array([[0.1, 0.4, 0.2, 0.3]] * 3, dtype=np.float32)
    u, rc = oracle.recalibrate(S, th, np.array([1, 2], dtype=np.uint32), 2)
    np.testing.assert_array_equal(u[0], [1.0, 0.5])
    np.testing.assert_array_equal(rc[0], np.array([0.4, 0.2], dtype=np.float32))
