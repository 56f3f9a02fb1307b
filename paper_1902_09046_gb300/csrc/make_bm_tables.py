"""Generates bm_tables.h, the tables of the table-driven Box-Muller in rng.cuh,
and checks the kernels' binary32 evaluation on every input the generator can
produce (2^23 uniforms per function).

The generator's uniforms are u = (m + 1/2) 2^-23, m = w >> 9 (23 bits), so
both functions of Box-Muller take one of 2^23 arguments:

  * -2 ln u, by the table-driven method of Tang (ACM TOMS 16(4), 1990):
    u = 2^e f with f in [3/4, 3/2) (the exponent split of u + 2^-2 ulp), the
    top 8 bits of f's field pick a bucket j, and with a table value c_j ~ 1/f
    r = f c_j - 1 is exact to one rounding, |r| <= 2^-9, and
        -2 ln u = e (-2 ln 2) + A_j - 2 log1p(r),   A_j = 2 ln c_j,
    -2 log1p(r) ~ t = -2 r + r^2 (1 - 2r/3) (truncation below 2^-29
    relative), summed as fma(e, K, A_j + t) with K = RN(-2 ln 2): e K is
    exact inside the fma, so only the add to A_j and the fma round; the
    error of K (3.8e-9) moves the result by at most |e| 3.8e-9, below 0.11
    ulp for every e (the f-range [3/4, 3/2) keeps -2 ln u >= 0.57 wherever
    e != 0).
    Each c_j is picked near the bucket centre so that 2 ln c_j lies within
    2^-12 ulp of a binary32 number (Gal's accurate tables, IBM, 1986), which
    makes the stored A_j almost exact; the bucket just below f = 1 takes
    c = 1, A = 0, so there r = f - 1 exactly and -2 ln u keeps full relative
    accuracy as u -> 1.
  * (cos, sin)(2 pi u): the angle index m splits as m = 2^11 i + k, so
    2 pi u = a_i + b_k with a_i = 2 pi i / 4096 and b_k = 2 pi (k + 1/2) 2^-23
    (|b_k| < 1.6e-3), and the angle-addition formulas combine a 4096-entry
    and a 2048-entry table:
        cos = C_i + (C_i cm_k - S_i s_k),  sin = S_i + (S_i cm_k + C_i s_k),
    with cm_k = cos b_k - 1 stored directly (it is about -1e-6, so storing
    cos b_k would round away most of it).

Every table value is the binary32 rounding of its exact value (mpmath at 60
digits).  `python make_bm_tables.py` rewrites bm_tables.h and prints the
worst-case errors over all 2^23 inputs of the binary32 evaluation above,
emulated with numpy (each fused multiply-add as one rounding of the exact
value, the product of two binary32 numbers being exact in binary64).
Nothing here runs at build or run time.
"""
import os

import mpmath
import numpy as np

mpmath.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "bm_tables.h")

LOG_BUCKETS = 256
SC_HI = 4096
SC_LO = 2048
K_HI = np.float32(-2 * np.log(2.0))


def f32(x):
    """binary32 rounding of an mpmath value (through binary64: exact for the
    magnitudes here unless the binary64 value sits on a binary32 tie, which
    is checked)."""
    d = float(x)
    r = np.float32(d)
    # the binary64 value must not sit within 1 binary64 ulp of a binary32 midpoint
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    for nb in (up, dn):
        mid = (float(r) + float(nb)) / 2
        assert abs(d - mid) > 4 * abs(np.spacing(d)) or d == float(r), (x, d, mid)
    return r


def bucket_centre(j):
    if j < 128:
        return mpmath.mpf(0.75) + (j + mpmath.mpf(0.5)) * mpmath.mpf(2) ** -9
    return 1 + (j - 128 + mpmath.mpf(0.5)) * mpmath.mpf(2) ** -8


def _near_float_error(c):
    """|2 ln c - RN32(2 ln c)| in ulps of the rounded value, for binary32 c
    (binary64 screening; accurate to about 2^-28 ulp)."""
    v = 2 * np.log(c.astype(np.float64))
    a = v.astype(np.float32)
    return np.abs(v - a.astype(np.float64)) / np.spacing(np.abs(a)).astype(np.float64)


def log_table():
    cs, As = [], []
    offs = np.arange(-30000, 30001, dtype=np.int64)
    order = np.argsort(np.abs(offs), kind="stable")
    for j in range(LOG_BUCKETS):
        if j == 127:  # f in [1 - 2^-9, 1): c = 1, A = 0
            cs.append(np.float32(1.0))
            As.append(np.float32(0.0))
            continue
        c0 = np.float32(float(1 / bucket_centre(j)))
        cand = (np.int64(c0.view(np.uint32)) + offs[order]).astype(np.uint32).view(np.float32)
        good = np.nonzero(_near_float_error(cand) < 2.0 ** -13)[0]
        for g in good:  # the candidate nearest the centre that passes at 60 digits
            c = cand[g]
            v = 2 * mpmath.log(mpmath.mpf(float(c)))
            a = np.float32(float(v))
            if abs(v - mpmath.mpf(float(a))) < mpmath.mpf(2) ** -12 * mpmath.mpf(float(np.spacing(abs(a)))):
                break
        else:
            raise AssertionError(f"no accurate-table point in bucket {j}")
        cs.append(c)
        As.append(a)
    return np.array(cs, np.float32), np.array(As, np.float32)


def sc_tables():
    hi = np.zeros((SC_HI, 2), np.float32)
    for i in range(SC_HI):
        a = 2 * mpmath.pi * i / SC_HI
        hi[i] = (f32(mpmath.cos(a)), f32(mpmath.sin(a)))
    lo = np.zeros((SC_LO, 2), np.float32)
    for k in range(SC_LO):
        b = 2 * mpmath.pi * (k + mpmath.mpf(0.5)) * mpmath.mpf(2) ** -23
        lo[k] = (f32(mpmath.cos(b) - 1), f32(mpmath.sin(b)))
    return hi, lo


# ---------------------------------------------------------------------------
# binary32 emulation of the kernels' evaluation
# ---------------------------------------------------------------------------

def _fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def _mul(a, b):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)).astype(np.float32)


def _add(a, b):
    return (np.asarray(a, np.float64) + np.asarray(b, np.float64)).astype(np.float32)


def emulate_neg2log(m, cs, As):
    u = ((m.astype(np.float64) + 0.5) * 2.0 ** -23).astype(np.float32)
    B = u.view(np.uint32).astype(np.int64)
    Bp = B + 0x00400000
    e = (Bp >> 23) - 127
    ef = e.astype(np.float32)
    f = (B - (Bp & 0xFF800000) + 0x3F800000).astype(np.uint32).view(np.float32)
    j = (Bp >> 15) & 0xFF
    c, A = cs[j], As[j]
    r = _fma(f, c, np.float32(-1))
    q = _fma(r, np.float32(-2.0 / 3.0), np.float32(1))
    rq = _mul(r, q)
    m2r = _mul(np.float32(-2), r)
    t = _fma(rq, r, m2r)
    return _fma(ef, K_HI, _add(A, t)), u


def emulate_sincos(m, hi, lo):
    i = m >> 11
    k = m & 0x7FF
    Ci, Si = hi[i, 0], hi[i, 1]
    cm, sk = lo[k, 0], lo[k, 1]
    c = _add(Ci, _fma(Ci, cm, -_mul(Si, sk)))
    s = _add(Si, _fma(Si, cm, _mul(Ci, sk)))
    return c, s


def check(cs, As, hi, lo):
    m = np.arange(2 ** 23, dtype=np.int64)
    L, u = emulate_neg2log(m, cs, As)
    ref = -2 * np.log((m + 0.5) * 2.0 ** -23)
    err_l = np.abs(L.astype(np.float64) - ref) / np.spacing(np.abs(L)).astype(np.float64)
    c, s = emulate_sincos(m, hi, lo)
    ang = 2 * np.pi * ((m + 0.5) * 2.0 ** -23)
    ec = np.abs(c.astype(np.float64) - np.cos(ang))
    es = np.abs(s.astype(np.float64) - np.sin(ang))
    rc = ec / np.spacing(np.maximum(np.abs(c), np.float32(2.0 ** -126))).astype(np.float64)
    rs = es / np.spacing(np.maximum(np.abs(s), np.float32(2.0 ** -126))).astype(np.float64)
    return {"neg2log_max_ulp": float(err_l.max()), "cos_max_abs": float(ec.max()),
            "sin_max_abs": float(es.max()), "cos_max_ulp": float(rc.max()), "sin_max_ulp": float(rs.max())}


def _hex(a):
    return ", ".join(f"0x{int(x):08x}u" for x in np.asarray(a, np.float32).view(np.uint32).ravel())


def write_header(cs, As, hi, lo):
    lines = [
        "// bm_tables.h -- written by make_bm_tables.py; do not edit.",
        "//",
        "// binary32 bit patterns of the table-driven Box-Muller (bm_table.cuh), as float2 entries:",
        "//   entries 0..4095     (cos, sin)(2 pi i / 4096);",
        "//   entries 4096..6143  (cos b_k - 1, sin b_k), b_k = 2 pi (k + 1/2) 2^-23;",
        "//   entries 6144..6399  (c_j, A_j = 2 ln c_j), j = 0..255, buckets of f in [3/4, 3/2).",
        "#pragma once",
        "",
        "#include <stdint.h>",
        "",
        "namespace ppabc {",
        "",
        f"constexpr int kBmLogBuckets = {LOG_BUCKETS};",
        f"constexpr int kBmScHi = {SC_HI};",
        f"constexpr int kBmScLo = {SC_LO};",
        f"constexpr uint32_t kBmLogK = 0x{int(np.float32(K_HI).view(np.uint32)):08x}u;  // RN(-2 ln 2)",
        "",
    ]
    flat = np.concatenate([np.asarray(a, np.float32).ravel() for a in (hi, lo, np.stack([cs, As], 1))])
    lines.append("// One array in the compact layout: the sin/cos tables, then the log table.")
    lines.append(f"__device__ const __align__(16) uint32_t kBmTablesBits[{flat.size}] = {{")
    for r0 in range(0, flat.size, 8):
        lines.append("    " + _hex(flat[r0:r0 + 8]) + ",")
    lines.append("};")
    lines.append("")
    lines.append("}  // namespace ppabc")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    cs, As = log_table()
    hi, lo = sc_tables()
    write_header(cs, As, hi, lo)
    for k, v in check(cs, As, hi, lo).items():
        print(f"{k}: {v:.4g}")


if __name__ == "__main__":
    main()
