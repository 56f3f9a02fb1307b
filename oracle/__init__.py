"""Plain FP64 CPU oracle for the prior-predictive Monte Carlo path.

TEST INFRASTRUCTURE ONLY.  This package wraps ``ppabc_oracle.c`` (plain C,
binary64, written from the paper and from the published Philox definition)
through ``ctypes``.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the product path never does, and the oracle
shares no code with the CUDA path.

Every function returns numpy arrays; see ``ppabc_oracle.h`` for the
conventions (counter layout, uniform and Box-Muller mapping).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppabc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_PRIOR = 0
TAG_PATH = 1
TAG_BASE = 2
TAG_TOGGLE_PRIOR = 4
TAG_TOGGLE_PATH = 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    srcs = [_SRC, os.path.join(_HERE, "ppabc_oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _ToggleModel(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 7), ("hi", ctypes.c_double * 7),
                ("T", ctypes.c_uint32), ("C", ctypes.c_uint32)]


class _OUModel(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("x0", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_steps", ctypes.c_uint32), ("n_obs", ctypes.c_uint32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, dbl, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
            lib.orc_philox_batch.argtypes = [u64, P, u64, P]
            lib.orc_philox_batch.restype = None
            lib.orc_u01.argtypes = [u32]
            lib.orc_u01.restype = dbl
            lib.orc_box_muller_words.argtypes = [P, u64, P]
            lib.orc_box_muller_words.restype = None
            lib.orc_stream_normals.argtypes = [u64, u32, u32, u32, u64, u64, P]
            lib.orc_stream_normals.restype = None
            lib.orc_ou_prior_predictive.argtypes = [ctypes.POINTER(_OUModel), P, u64, u64,
                                                    u64, u32, P, P, P, i32]
            lib.orc_ou_prior_predictive.restype = i32
            lib.orc_select_topk.argtypes = [P, u64, u64, P]
            lib.orc_select_topk.restype = i32
            lib.orc_select_eps.argtypes = [P, u64, dbl, P]
            lib.orc_select_eps.restype = u64
            lib.orc_moments.argtypes = [P, P, u64, P, P]
            lib.orc_moments.restype = None
            lib.orc_pvalue_sweep.argtypes = [P, u32, u32, u64, u64, dbl, u64, P, P, P, i32]
            lib.orc_pvalue_sweep.restype = i32
            lib.orc_weakinf.argtypes = [P, u32, dbl, u32, u64, dbl, u64, P, P, i32]
            lib.orc_weakinf.restype = i32
            lib.orc_toggle_prior_predictive.argtypes = [ctypes.POINTER(_ToggleModel), P, u64, u64,
                                                        u64, u32, P, P, P, P, P, i32]
            lib.orc_toggle_prior_predictive.restype = i32
            lib.orc_recalibrate.argtypes = [P, P, u64, u32, P, u64, u64, P, P, i32]
            lib.orc_recalibrate.restype = i32
            lib.orc_gammainc_p.argtypes = [dbl, dbl]
            lib.orc_gammainc_p.restype = dbl
            lib.orc_bege_cdf.argtypes = [dbl, dbl, dbl, dbl, dbl]
            lib.orc_bege_cdf.restype = dbl
            lib.orc_bege_density.argtypes = [dbl, dbl, dbl, dbl, dbl, dbl]
            lib.orc_bege_density.restype = dbl
            lib.orc_bege_loglik.argtypes = [P, u64, P, u32, dbl, P, P, i32]
            lib.orc_bege_loglik.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def philox(seed: int, ctr: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of each counter row (ctr: [n,4] uint32) -> [n,4] uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    _load().orc_philox_batch(seed, _ptr(ctr), ctr.shape[0], _ptr(out))
    return out


def u01(w: int) -> float:
    return _load().orc_u01(int(w) & 0xFFFFFFFF)


def box_muller_words(w: np.ndarray) -> np.ndarray:
    """Box-Muller normals of word pairs w [n,2] uint32 -> [n,2] float64."""
    w = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1, 2)
    z = np.zeros(w.shape, dtype=np.float64)
    _load().orc_box_muller_words(_ptr(w), w.shape[0], _ptr(z))
    return z


def stream_normals(seed: int, c1: int, c2: int, tag: int, j0: int, n: int) -> np.ndarray:
    z = np.zeros(n, dtype=np.float64)
    _load().orc_stream_normals(seed, c1, c2, tag, j0, n, _ptr(z))
    return z


def _model(lo, hi, x0, dt, n_steps, n_obs) -> _OUModel:
    m = _OUModel()
    for j in range(3):
        m.lo[j] = float(lo[j])
        m.hi[j] = float(hi[j])
    m.x0, m.dt, m.n_steps, m.n_obs = float(x0), float(dt), int(n_steps), int(n_obs)
    return m


def ou_prior_predictive(model: dict, y_obs, n: int, seed: int, sub: int = 0, base: int = 0,
                        want_theta: bool = True, want_summ: bool = False,
                        n_threads: int | None = None):
    """(theta [n,3] | None, summ [n,n_obs] | None, dist [n]) for samples base..base+n-1."""
    m = _model(model["lo"], model["hi"], model.get("x0", 0.0), model["dt"],
               model["n_steps"], model["n_obs"])
    y = np.ascontiguousarray(y_obs, dtype=np.float64)
    if y.shape[0] != m.n_obs:
        raise ValueError("y_obs length must equal n_obs")
    theta = np.zeros((n, 3), dtype=np.float64) if want_theta else None
    summ = np.zeros((n, m.n_obs), dtype=np.float64) if want_summ else None
    dist = np.zeros(n, dtype=np.float64)
    rc = _load().orc_ou_prior_predictive(ctypes.byref(m), _ptr(y), base, n, seed, sub,
                                         _ptr(theta), _ptr(summ), _ptr(dist),
                                         n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle rejected the OU arguments")
    return theta, summ, dist


def select_topk(dist: np.ndarray, k: int) -> np.ndarray:
    d = np.ascontiguousarray(dist, dtype=np.float64)
    idx = np.zeros(max(k, 1), dtype=np.uint64)
    if _load().orc_select_topk(_ptr(d), d.shape[0], k, _ptr(idx)) != 0:
        raise ValueError("k > n")
    return idx[:k]


def select_eps(dist: np.ndarray, eps: float) -> np.ndarray:
    d = np.ascontiguousarray(dist, dtype=np.float64)
    idx = np.zeros(max(d.shape[0], 1), dtype=np.uint64)
    c = _load().orc_select_eps(_ptr(d), d.shape[0], float(eps), _ptr(idx))
    return idx[:c]


def moments(theta: np.ndarray, idx: np.ndarray):
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 3)
    ix = np.ascontiguousarray(idx, dtype=np.uint64)
    mean = np.zeros(3)
    var = np.zeros(3)
    _load().orc_moments(_ptr(th), _ptr(ix), ix.shape[0], _ptr(mean), _ptr(var))
    return mean, var


def pvalue_sweep(lambdas, n_obs: int, m_sets: int, ybar_obs: float, seed: int,
                 want_ybar: bool = False, n_threads: int | None = None, base: int = 0):
    """(counts [K] uint64, p [K], ybar [K,M] | None)."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    K = lam.shape[0]
    counts = np.zeros(K, dtype=np.uint64)
    p = np.zeros(K, dtype=np.float64)
    ybar = np.zeros((K, m_sets), dtype=np.float64) if want_ybar else None
    rc = _load().orc_pvalue_sweep(_ptr(lam), K, n_obs, m_sets, base, float(ybar_obs), seed,
                                  _ptr(counts), _ptr(p), _ptr(ybar),
                                  n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle rejected the p-value arguments")
    return counts, p, ybar


def weakinf(lambdas, lambda0: float, n_obs: int, n_sets: int, alpha: float, seed: int,
            want_counts: bool = False, n_threads: int | None = None):
    """(gamma [K], counts [K,N] | None): Algorithm 2's alpha-level cut-offs."""
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    K = lam.shape[0]
    gamma = np.zeros(K, dtype=np.float64)
    counts = np.zeros((K, n_sets), dtype=np.uint64) if want_counts else None
    rc = _load().orc_weakinf(_ptr(lam), K, float(lambda0), n_obs, n_sets, float(alpha), seed,
                             _ptr(gamma), _ptr(counts), n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle rejected the weak-informativity arguments")
    return gamma, counts


def toggle_prior_predictive(model: dict, q_obs, n: int, seed: int, sub: int = 0, base: int = 0,
                            want_theta: bool = True, want_summ: bool = True, want_y: bool = False,
                            n_threads: int | None = None, want_uv: bool = False):
    """(theta [n,7], summ [n,19], y [n,C] | None, dist [n]) of the toggle-switch model;
    with want_uv a fifth item, the final (u, v) of every cell [n,C,2]."""
    m = _ToggleModel()
    for j in range(7):
        m.lo[j] = float(model["lo"][j])
        m.hi[j] = float(model["hi"][j])
    m.T, m.C = int(model["T"]), int(model["C"])
    q = np.ascontiguousarray(q_obs, dtype=np.float64)
    theta = np.zeros((n, 7)) if want_theta else None
    summ = np.zeros((n, 19)) if want_summ else None
    y = np.zeros((n, m.C)) if want_y else None
    uv = np.zeros((n, m.C, 2)) if want_uv else None
    dist = np.zeros(n)
    rc = _load().orc_toggle_prior_predictive(ctypes.byref(m), _ptr(q), base, n, seed, sub,
                                             _ptr(theta), _ptr(summ), _ptr(y), _ptr(uv),
                                             _ptr(dist), n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle rejected the toggle-switch arguments")
    if want_uv:
        return theta, summ, y, dist, uv
    return theta, summ, y, dist


def recalibrate(summ: np.ndarray, theta: np.ndarray, acc: np.ndarray, k: int,
                n_threads: int | None = None):
    """ABC recalibration: summ [n_obs, n] float64, theta [3, n] float32, acc [q]
    accepted indices -> (u [3, q] float64, theta_rc [3, q] float32)."""
    S = np.ascontiguousarray(summ, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float32)
    a = np.ascontiguousarray(acc, dtype=np.uint32)
    n_obs, n = S.shape
    q = a.shape[0]
    u = np.zeros((3, q), dtype=np.float64)
    rc_out = np.zeros((3, q), dtype=np.float32)
    rc = _load().orc_recalibrate(_ptr(S), _ptr(th), n, n_obs, _ptr(a), q, k, _ptr(u), _ptr(rc_out),
                                 n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle rejected the recalibration arguments")
    return u, rc_out


BEGE_NPAR = 11
BEGE_NW = 100
BEGE_PARAMS = ("p0", "sigma_p", "rho_p", "phi_p_plus", "phi_p_minus",
               "n0", "sigma_n", "rho_n", "phi_n_plus", "phi_n_minus", "mu")


def gammainc_p(a, x) -> np.ndarray:
    """Regularised lower incomplete gamma P(a, x), elementwise."""
    A, X = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(x, dtype=np.float64))
    f = _load().orc_gammainc_p
    return np.array([f(float(ai), float(xi)) for ai, xi in zip(A.ravel(), X.ravel())]).reshape(A.shape)


def bege_cdf(u, sp: float, sn: float, p: float, n: float) -> np.ndarray:
    """The discretised BEGE distribution function at each u."""
    f = _load().orc_bege_cdf
    U = np.asarray(u, dtype=np.float64)
    return np.array([f(float(v), sp, sn, p, n) for v in U.ravel()]).reshape(U.shape)


def bege_density(u, sp: float, sn: float, p: float, n: float, h: float) -> np.ndarray:
    """The BEGE density at each u by central differences with step h."""
    f = _load().orc_bege_density
    U = np.asarray(u, dtype=np.float64)
    return np.array([f(float(v), sp, sn, p, n, h) for v in U.ravel()]).reshape(U.shape)


def bege_loglik(theta: np.ndarray, r: np.ndarray, h: float, want_dens: bool = False,
                n_threads: int | None = None):
    """theta [11, np] float64 (rows in BEGE_PARAMS order), r [T] -> ll [np]
    (and, with want_dens, the densities [np, T])."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    if th.ndim != 2 or th.shape[0] != BEGE_NPAR:
        raise ValueError("theta must be [11, np]")
    n_p, T = th.shape[1], rr.shape[0]
    ll = np.zeros(n_p)
    dens = np.zeros((n_p, T)) if want_dens else None
    rc = _load().orc_bege_loglik(_ptr(th), n_p, _ptr(rr), T, h, _ptr(ll), _ptr(dens),
                                 n_threads or default_threads())
    if rc != 0:
        raise ValueError("oracle rejected the BEGE arguments")
    return (ll, dens) if want_dens else ll
