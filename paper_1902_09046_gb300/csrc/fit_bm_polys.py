"""Derives the binary32 polynomial coefficients used by rng.cuh's Box-Muller.

Both polynomials are fitted here from the mathematics (iteratively reweighted
least squares on Chebyshev nodes, converging to a near-minimax relative
error), rounded to binary32, and then checked by emulating the kernels'
binary32 Horner evaluation on EVERY input the generator can produce (2^23
uniforms), against binary64 references:

  * -2 ln(u), u = (m + 1/2) 2^-23:  reduce u = 2^e f, f in [sqrt(1/2), sqrt(2)),
    s = f - 1, then -2 ln u = e (-2 ln 2) + (-2 s + s^2 Q(s)) with Q of degree 8;
  * sin(pi t), cos(pi t), |t| <= 1/4 (after an exact quadrant reduction of
    2u): sin = fma(t, pi_hi, t (pi_lo + t^2 P(t^2))), cos = 1 + t^2 R(t^2).

Run `python fit_bm_polys.py` to print the coefficients and their worst-case
errors in ulp.  numpy only; nothing here runs at build or run time.
"""
import numpy as np


def _irls(x, y, basis, base, n_iter=80):
    A = np.stack([b(x) for b in basis], 1)
    w = np.ones_like(x)
    for _ in range(n_iter):
        W = w / np.abs(y)
        c, *_ = np.linalg.lstsq(A * W[:, None], (y - base) * W, rcond=None)
        err = np.abs(base + A @ c - y) / np.abs(y)
        w = w * (err / err.max()) ** 0.3 + 1e-14
    return c


def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(np.float32)


def _cheb(lo, hi, n):
    return np.cos(np.linspace(0, np.pi, n)) * (hi - lo) / 2 + (hi + lo) / 2


def fit_log():
    lo, hi = np.sqrt(0.5) - 1, np.sqrt(2) - 1
    x = _cheb(lo, hi, 20000)
    x = x[np.abs(x) > 1e-6]
    y = -2 * np.log1p(x)
    c = _irls(x, y, [(lambda k: (lambda s: s ** (k + 2)))(k) for k in range(9)], -2 * x)
    return [np.float32(v) for v in c]


def check_log(Q):
    m = np.arange(2 ** 23, dtype=np.float64)
    u = ((m + 0.5) * 2.0 ** -23).astype(np.float32)
    v = u.view(np.uint32).astype(np.int64)
    e = (v - 0x3F3504F3) >> 23
    f = (v - (e << 23)).astype(np.uint32).view(np.float32)
    s = (f - np.float32(1)).astype(np.float32)
    q = np.full_like(s, Q[-1])
    for cc in Q[-2::-1]:
        q = _fma(q, s, cc)
    t = _fma((s * s).astype(np.float32), q, (np.float32(-2) * s).astype(np.float32))
    h2 = np.float32(-2 * np.log(2.0))
    l2 = np.float32(-2 * np.log(2.0) - np.float64(h2))
    ef = e.astype(np.float32)
    L = _fma(ef, h2, _fma(ef, l2, t))
    ref = -2 * np.log((m + 0.5) * 2.0 ** -23)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    return float(np.max(np.abs(L - ref) / ulp)), h2, l2


def fit_sincos():
    x = _cheb(0, 0.25, 8000)
    x = x[x > 1e-7]
    pi_hi = np.float32(np.pi)
    pi_lo = np.float32(np.pi - np.float64(pi_hi))
    S = _irls(x, np.sin(np.pi * x), [lambda t: t ** 3, lambda t: t ** 5, lambda t: t ** 7], np.pi * x)
    C = _irls(x, np.cos(np.pi * x), [lambda t: t ** 2, lambda t: t ** 4, lambda t: t ** 6,
                                     lambda t: t ** 8], np.ones_like(x))
    return pi_hi, pi_lo, [np.float32(v) for v in S], [np.float32(v) for v in C]


def check_sincos(pi_hi, pi_lo, S, C):
    t = (np.arange(1, 2 ** 21 + 1, dtype=np.float64) * 2 - 1) * 2.0 ** -23
    t = t[t <= 0.25]
    t32 = t.astype(np.float32)
    t2 = (t32 * t32).astype(np.float32)
    ps = _fma(_fma(_fma(np.full_like(t2, S[2]), t2, S[1]), t2, S[0]), t2, pi_lo)
    s = _fma(t32, pi_hi, (t32 * ps).astype(np.float32))
    pc = _fma(_fma(_fma(np.full_like(t2, C[3]), t2, C[2]), t2, C[1]), t2, C[0])
    c = _fma(pc, t2, np.float32(1))
    ulp = lambda r: np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)
    rs, rc = np.sin(np.pi * t), np.cos(np.pi * t)
    return float(np.max(np.abs(s - rs) / ulp(rs))), float(np.max(np.abs(c - rc) / ulp(rc)))


if __name__ == "__main__":
    Q = fit_log()
    err, h2, l2 = check_log(Q)
    print("log: Q =", [repr(float(v)) for v in Q])
    print(f"     -2 ln2 = {float(h2)!r} + {float(l2)!r}; max error over all inputs {err:.3f} ulp")
    pi_hi, pi_lo, S, C = fit_sincos()
    es, ec = check_sincos(pi_hi, pi_lo, S, C)
    print("sin: pi =", repr(float(pi_hi)), "+", repr(float(pi_lo)), "; P =", [repr(float(v)) for v in S])
    print("cos: R =", [repr(float(v)) for v in C])
    print(f"     max error over all inputs: sin {es:.3f} ulp, cos {ec:.3f} ulp")
