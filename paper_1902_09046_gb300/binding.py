"""Thin Python binding of libppabc.so (argument marshalling only).

Each function has the name of the C entry point it calls (see
``include/ppabc.h``), takes and returns torch tensors on the current CUDA
device, and enqueues work on the current torch stream (or ``stream``).  All
computation happens in the library's CUDA kernels; if the library is not
built or no sm_103 device is current, calls raise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

from . import build as _build

PPABC_OK = 0
PPABC_EINVAL = -1
PPABC_ENOMEM = -2
PPABC_ECUDA = -3
PPABC_ETIMEOUT = -4
PPABC_ENODEV = -5
PPABC_ECANCELLED = -6
PPABC_MAX_OBS = 32
TAG_PRIOR = 0
TAG_PATH = 1

_ERRNAMES = {PPABC_EINVAL: "EINVAL", PPABC_ENOMEM: "ENOMEM", PPABC_ECUDA: "ECUDA",
             PPABC_ETIMEOUT: "ETIMEOUT", PPABC_ENODEV: "ENODEV", PPABC_ECANCELLED: "ECANCELLED"}

# Every symbol include/ppabc.h declares (checked by the CPU test-suite).
EXPORTED = ("ppabc_abi_version", "ppabc_last_error", "ppabc_device_check", "ppabc_philox_raw",
            "ppabc_normals", "abc_prior_predictive", "abc_select_workspace_bytes", "abc_select",
            "abc_select_static", "pvalue_sweep")
STATIC_SELECT_MAX_N = 1 << 24


class PPABCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ppabc {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class OUModel(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("x0", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_steps", ctypes.c_uint32), ("n_obs", ctypes.c_uint32)]

    @classmethod
    def from_dict(cls, m: dict) -> "OUModel":
        o = cls()
        for j in range(3):
            o.lo[j] = float(m["lo"][j])
            o.hi[j] = float(m["hi"][j])
        o.x0 = float(m.get("x0", 0.0))
        o.dt = float(m["dt"])
        o.n_steps = int(m["n_steps"])
        o.n_obs = int(m["n_obs"])
        return o


_lock = threading.Lock()
_lib_handle = None


def library_path() -> str:
    return _build.LIB_PATH


def load_library(build_if_missing: bool = False) -> ctypes.CDLL:
    """Loads libppabc.so (without touching the GPU)."""
    global _lib_handle
    with _lock:
        if _lib_handle is not None:
            return _lib_handle
        path = _build.LIB_PATH
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_1902_09046_gb300.build`")
            _build.build()
        lib = ctypes.CDLL(path)
        P, u32, u64, dbl, i32, sz = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_size_t)
        M = ctypes.POINTER(OUModel)
        sig = {
            "ppabc_abi_version": ([], i32),
            "ppabc_last_error": ([], ctypes.c_char_p),
            "ppabc_device_check": ([], i32),
            "ppabc_philox_raw": ([u64, P, u64, P, P], i32),
            "ppabc_normals": ([u64, u32, u32, u32, u64, u64, P, P], i32),
            "abc_prior_predictive": ([M, P, u64, u64, u64, u32, P, P, P, P], i32),
            "abc_select_workspace_bytes": ([u64], sz),
            "abc_select": ([P, u64, u64, dbl, M, u64, u64, u32, P, P, P, u64, P, P, P, P, sz, P], i32),
            "abc_select_static": ([P, u64, u64, dbl, M, u64, u64, u32, P, P, P, u64, P, P, P, P], i32),
            "pvalue_sweep": ([P, u32, u32, u64, u64, dbl, u64, P, P, P, P], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib_handle = lib
        return lib


def _check(rc: int) -> None:
    if rc != PPABC_OK:
        msg = load_library().ppabc_last_error().decode(errors="replace")
        raise PPABCError(rc, msg)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def device_check() -> None:
    _check(load_library().ppabc_device_check())


def philox_raw(seed: int, ctr: torch.Tensor, stream=None) -> torch.Tensor:
    """ctr: [n,4] uint32 (CUDA) -> [n,4] uint32 Philox4x32-10 blocks."""
    if ctr.dtype != torch.uint32 or ctr.dim() != 2 or ctr.shape[1] != 4:
        raise ValueError("ctr must be a [n,4] uint32 tensor")
    out = torch.empty_like(ctr)
    _check(load_library().ppabc_philox_raw(seed, _ptr(ctr), ctr.shape[0], _ptr(out), _stream(stream)))
    return out


def normals(seed: int, c1: int, c2: int, tag: int, j0: int, n: int, stream=None) -> torch.Tensor:
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(load_library().ppabc_normals(seed, c1, c2, tag, j0, n, _ptr(z), _stream(stream)))
    return z


def _y_obs_host(y_obs) -> ctypes.Array:
    vals = [float(v) for v in (y_obs.tolist() if hasattr(y_obs, "tolist") else y_obs)]
    return (ctypes.c_double * max(1, len(vals)))(*vals)


def abc_prior_predictive(model: dict, y_obs, n_samples: int, seed: int, substream: int = 0,
                         sample_base: int = 0, want_theta: bool = True, want_summ: bool = False,
                         out: dict | None = None, stream=None) -> dict:
    """Returns {"theta": [3,N] f32 | None, "summ": [n_obs,N] f64 | None, "dist": [N] f64}."""
    m = OUModel.from_dict(model)
    out = dict(out or {})
    dev = torch.device("cuda")
    dist = out.get("dist")
    if dist is None:
        dist = torch.empty(n_samples, dtype=torch.float64, device=dev)
    theta = out.get("theta")
    if want_theta and theta is None:
        theta = torch.empty((3, n_samples), dtype=torch.float32, device=dev)
    summ = out.get("summ")
    if want_summ and summ is None:
        summ = torch.empty((m.n_obs, n_samples), dtype=torch.float64, device=dev)
    y = _y_obs_host(y_obs)
    _check(load_library().abc_prior_predictive(ctypes.byref(m), y, n_samples, sample_base, seed,
                                               substream, _ptr(theta if want_theta else None),
                                               _ptr(summ if want_summ else None), _ptr(dist),
                                               _stream(stream)))
    return {"theta": theta if want_theta else None, "summ": summ if want_summ else None,
            "dist": dist}


def abc_select_workspace_bytes(n: int) -> int:
    return int(load_library().abc_select_workspace_bytes(n))


def abc_select(dist: torch.Tensor, k: int = 0, eps: float = math.inf, model: dict | None = None,
               seed: int = 0, substream: int = 0, sample_base: int = 0,
               theta: torch.Tensor | None = None, cap: int | None = None,
               workspace: torch.Tensor | None = None, out: dict | None = None,
               stream=None) -> dict:
    """k > 0: the k nearest; k = 0: all with dist <= eps.  Returns tensors
    idx [cap] u32, rec [cap,4] f32, n_acc [1] u64, eps [1] f64, post [6] f64."""
    n = dist.shape[0]
    if cap is None:
        cap = k if k > 0 else n
    dev = dist.device
    out = dict(out or {})
    idx = out.get("idx")
    if idx is None:
        idx = torch.empty(max(cap, 1), dtype=torch.uint32, device=dev)
    rec = out.get("rec")
    if rec is None:
        rec = torch.empty((max(cap, 1), 4), dtype=torch.float32, device=dev)
    n_acc = out.get("n_acc")
    if n_acc is None:
        n_acc = torch.empty(1, dtype=torch.uint64, device=dev)
    eps_t = out.get("eps")
    if eps_t is None:
        eps_t = torch.empty(1, dtype=torch.float64, device=dev)
    post = out.get("post")
    if post is None:
        post = torch.empty(6, dtype=torch.float64, device=dev)
    lib = load_library()
    ws_bytes = int(lib.abc_select_workspace_bytes(n))
    if workspace is None:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    mdl = ctypes.byref(OUModel.from_dict(model)) if model is not None else None
    _check(lib.abc_select(_ptr(dist), n, k, float(eps), mdl, sample_base, seed, substream,
                          _ptr(theta), _ptr(idx), _ptr(rec), cap, _ptr(n_acc), _ptr(eps_t),
                          _ptr(post), _ptr(workspace), workspace.numel() * workspace.element_size(),
                          _stream(stream)))
    return {"idx": idx[:cap], "rec": rec[:cap], "n_acc": n_acc, "eps": eps_t, "post": post}


def abc_select_static(dist: torch.Tensor, k: int = 0, eps: float = math.inf,
                      model: dict | None = None, seed: int = 0, substream: int = 0,
                      sample_base: int = 0, theta: torch.Tensor | None = None,
                      cap: int | None = None, out: dict | None = None, stream=None) -> dict:
    """abc_select whose scratch is the library's static device array: for
    callers that cannot allocate device memory.  At most STATIC_SELECT_MAX_N
    distances; calls that overlap on the GPU race on the shared scratch.
    The output tensors are allocated here unless passed in ``out``."""
    n = dist.shape[0]
    if cap is None:
        cap = k if k > 0 else n
    dev = dist.device
    out = dict(out or {})
    res = {"idx": out.get("idx"), "rec": out.get("rec"), "n_acc": out.get("n_acc"),
           "eps": out.get("eps"), "post": out.get("post")}
    shapes = {"idx": ((max(cap, 1),), torch.uint32), "rec": ((max(cap, 1), 4), torch.float32),
              "n_acc": ((1,), torch.uint64), "eps": ((1,), torch.float64),
              "post": ((6,), torch.float64)}
    for key, (shape, dtype) in shapes.items():
        if res[key] is None:
            res[key] = torch.empty(shape, dtype=dtype, device=dev)
    mdl = ctypes.byref(OUModel.from_dict(model)) if model is not None else None
    _check(load_library().abc_select_static(
        _ptr(dist), n, k, float(eps), mdl, sample_base, seed, substream, _ptr(theta),
        _ptr(res["idx"]), _ptr(res["rec"]), cap, _ptr(res["n_acc"]), _ptr(res["eps"]),
        _ptr(res["post"]), _stream(stream)))
    res["idx"] = res["idx"][:cap]
    res["rec"] = res["rec"][:cap]
    return res


def pvalue_sweep(lambdas: torch.Tensor, n_obs: int, m_sets: int, ybar_obs: float, seed: int,
                 want_ybar: bool = False, set_base: int = 0, out: dict | None = None,
                 stream=None) -> dict:
    """lambdas: [K] f64 (CUDA).  Returns counts [K] u64, p [K] f64, ybar [K,M] f64 | None."""
    K = lambdas.shape[0]
    dev = lambdas.device
    out = dict(out or {})
    counts = out.get("counts")
    if counts is None:
        counts = torch.empty(K, dtype=torch.uint64, device=dev)
    p = out.get("p")
    if p is None:
        p = torch.empty(K, dtype=torch.float64, device=dev)
    ybar = out.get("ybar")
    if want_ybar and ybar is None:
        ybar = torch.empty((K, m_sets), dtype=torch.float64, device=dev)
    _check(load_library().pvalue_sweep(_ptr(lambdas), K, n_obs, m_sets, set_base, float(ybar_obs), seed,
                                       _ptr(counts), _ptr(p), _ptr(ybar if want_ybar else None),
                                       _stream(stream)))
    return {"counts": counts, "p": p, "ybar": ybar if want_ybar else None}
