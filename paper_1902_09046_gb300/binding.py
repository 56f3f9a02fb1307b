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
EXPORTED = ("ppabc_abi_version", "ppabc_last_error", "ppabc_device_check", "ppabc_device_info", "ppabc_philox_raw",
            "ppabc_normals", "ppabc_box_muller", "abc_prior_predictive", "abc_select_workspace_bytes", "abc_select",
            "abc_select_static", "abc_select_candidates", "abc_merge_workspace_bytes", "abc_merge_candidates",
            "pvalue_sweep", "ppabc_batch_workspace_bytes",
            "ppabc_batch_prepare", "ppabc_batch_launch", "ppabc_batch_launch_graph",
            "ppabc_batch_plan_destroy", "ppabc_batch_run", "ppabc_server_create",
            "ppabc_server_submit", "ppabc_server_poll", "ppabc_server_wait", "ppabc_server_fetch",
            "ppabc_server_release", "ppabc_server_cancel", "ppabc_server_get_stats",
            "ppabc_server_now", "ppabc_server_destroy", "weakinf_test_workspace_bytes", "weakinf_test",
            "toggle_prior_predictive",
            "abc_rejection_workspace_bytes", "abc_rejection", "abc_recalibrate_workspace_bytes",
            "abc_recalibrate", "bege_loglik_workspace_bytes", "bege_loglik")
WEAKINF_MAX_SETS = 16384
PPABC_PENDING = 1
JOB_ABC = 0
JOB_PVALUE = 1
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


class ABCJob(ctypes.Structure):
    _fields_ = [("model", OUModel), ("y_obs", ctypes.c_double * PPABC_MAX_OBS),
                ("n_samples", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("substream", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("k", ctypes.c_uint64), ("eps", ctypes.c_double),
                ("dist", ctypes.c_void_p), ("idx_out", ctypes.c_void_p),
                ("rec_out", ctypes.c_void_p), ("cap", ctypes.c_uint64),
                ("n_acc_out", ctypes.c_void_p), ("eps_out", ctypes.c_void_p),
                ("post_out", ctypes.c_void_p)]


class ToggleModel(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 7), ("hi", ctypes.c_double * 7),
                ("T", ctypes.c_uint32), ("C", ctypes.c_uint32)]

    @classmethod
    def from_dict(cls, m: dict) -> "ToggleModel":
        o = cls()
        for j in range(7):
            o.lo[j] = float(m["lo"][j])
            o.hi[j] = float(m["hi"][j])
        o.T, o.C = int(m["T"]), int(m["C"])
        return o


class TileConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("min_tile_steps", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("substream", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("model", OUModel), ("y_obs", ctypes.c_double * PPABC_MAX_OBS),
                ("n_samples", ctypes.c_uint64), ("k", ctypes.c_uint64), ("lam", ctypes.c_double),
                ("n_obs", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("m_sets", ctypes.c_uint64), ("ybar_obs", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("job_id", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("n_acc", ctypes.c_uint64), ("eps", ctypes.c_double),
                ("post", ctypes.c_double * 6), ("count", ctypes.c_uint64), ("p", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"status": self.status, "kind": self.kind, "job_id": self.job_id,
                "t_submit": self.t_submit, "t_admit": self.t_admit, "t_done": self.t_done,
                "n_acc": self.n_acc, "eps": self.eps, "post": list(self.post),
                "count": self.count, "p": self.p}


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "failed",
                                               "cancelled", "queued", "running",
                                               "arena_used_bytes", "peak_arena_bytes")]


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
            "ppabc_device_info": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], i32),
            "ppabc_philox_raw": ([u64, P, u64, P, P], i32),
            "ppabc_normals": ([u64, u32, u32, u32, u64, u64, u32, P, P], i32),
            "ppabc_box_muller": ([P, u64, u32, P, P], i32),
            "abc_prior_predictive": ([M, P, u64, u64, u64, u32, P, P, P, P], i32),
            "abc_select_workspace_bytes": ([u64], sz),
            "abc_select": ([P, u64, u64, dbl, M, u64, u64, u32, P, P, P, u64, P, P, P, P, sz, P], i32),
            "abc_select_static": ([P, u64, u64, dbl, M, u64, u64, u32, P, P, P, u64, P, P, P, P], i32),
            "abc_select_candidates": ([P, u64, u64, P, P, u64, P, P, P, P], i32),
            "abc_merge_workspace_bytes": ([u64, u64], sz),
            "abc_merge_candidates": ([P, P, P, u64, u64, P, P, P, P, P, P, sz, P], i32),
            "pvalue_sweep": ([P, u32, u32, u64, u64, dbl, u64, P, P, P, P], i32),
            "ppabc_batch_workspace_bytes": ([P, u32], sz),
            "ppabc_batch_prepare": ([P, u32, P, P, sz, P, ctypes.POINTER(P)], i32),
            "ppabc_batch_launch": ([P, P], i32),
            "ppabc_batch_launch_graph": ([P, P], i32),
            "ppabc_batch_plan_destroy": ([P], i32),
            "ppabc_batch_run": ([P, u32, P, P, sz, P], i32),
            "ppabc_server_create": ([P, sz, u32, ctypes.POINTER(P)], i32),
            "ppabc_server_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(u64)], i32),
            "ppabc_server_poll": ([P, u64, ctypes.POINTER(Result)], i32),
            "ppabc_server_wait": ([P, u64, dbl, ctypes.POINTER(Result)], i32),
            "ppabc_server_fetch": ([P, u64, P, P, u64, ctypes.POINTER(u64)], i32),
            "ppabc_server_release": ([P, u64], i32),
            "ppabc_server_cancel": ([P, u64], i32),
            "ppabc_server_get_stats": ([P, ctypes.POINTER(ServerStats)], i32),
            "ppabc_server_now": ([P], dbl),
            "ppabc_server_destroy": ([P], i32),
            "weakinf_test_workspace_bytes": ([u64, u64], sz),
            "weakinf_test": ([P, u32, dbl, u32, u64, dbl, u64, P, P, P, sz, P], i32),
            "abc_rejection_workspace_bytes": ([u64], sz),
            "abc_rejection": ([M, P, dbl, u64, u64, u64, u64, u32, P, P, P, P, sz, P], i32),
            "abc_recalibrate_workspace_bytes": ([u64, u64], sz),
            "abc_recalibrate": ([P, P, u64, u32, P, u64, u64, P, P, P, sz, P], i32),
            "bege_loglik_workspace_bytes": ([u64, u32], sz),
            "bege_loglik": ([P, u64, P, u32, dbl, P, P, P, sz, P], i32),
            "toggle_prior_predictive": ([ctypes.POINTER(ToggleModel), P, u64, u64, u64, u32, P, P,
                                         P, P, P], i32),
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


def device_info() -> tuple[int, float]:
    """(SM count, maximum SM clock in MHz) of the current device."""
    sms, khz = ctypes.c_int(0), ctypes.c_int(0)
    _check(load_library().ppabc_device_info(ctypes.byref(sms), ctypes.byref(khz)))
    return sms.value, khz.value / 1e3


def philox_raw(seed: int, ctr: torch.Tensor, stream=None) -> torch.Tensor:
    """ctr: [n,4] uint32 (CUDA) -> [n,4] uint32 Philox4x32-10 blocks."""
    if ctr.dtype != torch.uint32 or ctr.dim() != 2 or ctr.shape[1] != 4:
        raise ValueError("ctr must be a [n,4] uint32 tensor")
    out = torch.empty_like(ctr)
    _check(load_library().ppabc_philox_raw(seed, _ptr(ctr), ctr.shape[0], _ptr(out), _stream(stream)))
    return out


BM_POLY = 0
BM_TABLE = 1


def normals(seed: int, c1: int, c2: int, tag: int, j0: int, n: int, method: int = BM_TABLE,
            stream=None) -> torch.Tensor:
    """Normals j0..j0+n-1 of stream (index c1, substream c2, tag) by the
    Box-Muller evaluation `method` (BM_TABLE: the OU path kernels', BM_POLY:
    the p-value, Algorithm 2 and toggle kernels')."""
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(load_library().ppabc_normals(seed, c1, c2, tag, j0, n, method, _ptr(z), _stream(stream)))
    return z


def box_muller(w: torch.Tensor, method: int = BM_TABLE, stream=None) -> torch.Tensor:
    """w: [n,2] uint32 (CUDA) -> [n,2] float32 Box-Muller normals."""
    if w.dtype != torch.uint32 or w.dim() != 2 or w.shape[1] != 2:
        raise ValueError("w must be a [n,2] uint32 tensor")
    z = torch.empty(w.shape, dtype=torch.float32, device=w.device)
    _check(load_library().ppabc_box_muller(_ptr(w), w.shape[0], method, _ptr(z), _stream(stream)))
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


def abc_select_candidates(dist: torch.Tensor, sel: dict, count: int, sample_base: int = 0,
                          stream=None) -> dict:
    """This rank's accepted samples (abc_select's output `sel` on `dist`) as a
    candidate record for the merge: {"dist": [count] f64, "index": [count]
    u64 global indices, "theta": [3,count] f32}."""
    dev = dist.device
    cand = {"dist": torch.empty(max(count, 1), dtype=torch.float64, device=dev),
            "index": torch.empty(max(count, 1), dtype=torch.uint64, device=dev),
            "theta": torch.empty((3, max(count, 1)), dtype=torch.float32, device=dev)}
    _check(load_library().abc_select_candidates(_ptr(dist), dist.shape[0], sample_base, _ptr(sel["idx"]),
                                                _ptr(sel["rec"]), count, _ptr(cand["dist"]),
                                                _ptr(cand["index"]), _ptr(cand["theta"]), _stream(stream)))
    return {"dist": cand["dist"][:count], "index": cand["index"][:count],
            "theta": cand["theta"][:, :count] if count else cand["theta"][:, :0]}


def abc_merge_candidates(cand_dist: torch.Tensor, cand_index: torch.Tensor, cand_theta: torch.Tensor,
                         k: int, stream=None) -> dict:
    """The k nearest of gathered candidates (concatenated in rank order):
    {"idx": [k] u64 global indices, "rec": [k,4] f32, "n_acc", "eps", "post"}."""
    m = cand_dist.shape[0]
    dev = cand_dist.device
    theta = cand_theta.contiguous()
    out = {"idx": torch.empty(k, dtype=torch.uint64, device=dev),
           "rec": torch.empty((k, 4), dtype=torch.float32, device=dev),
           "n_acc": torch.empty(1, dtype=torch.uint64, device=dev),
           "eps": torch.empty(1, dtype=torch.float64, device=dev),
           "post": torch.empty(6, dtype=torch.float64, device=dev)}
    lib = load_library()
    ws_bytes = int(lib.abc_merge_workspace_bytes(m, k))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    _check(lib.abc_merge_candidates(_ptr(cand_dist), _ptr(cand_index), _ptr(theta), m, k, _ptr(out["idx"]),
                                    _ptr(out["rec"]), _ptr(out["n_acc"]), _ptr(out["eps"]), _ptr(out["post"]),
                                    _ptr(ws), ws_bytes, _stream(stream)))
    return out


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


def abc_rejection(model: dict, y_obs, eps: float, m_accept: int, max_samples: int, seed: int,
                  chunk: int = 1 << 20, substream: int = 0, stream=None) -> dict:
    """Algorithm 1: the first m_accept proposals with rho <= eps.  Returns
    {"idx": [n_acc] u32, "rec": [n_acc,4] f32, "n_acc": int, "tried": int}."""
    m = OUModel.from_dict(model)
    dev = torch.device("cuda")
    idx = torch.empty(m_accept, dtype=torch.uint32, device=dev)
    rec = torch.empty((m_accept, 4), dtype=torch.float32, device=dev)
    lib = load_library()
    ws_bytes = int(lib.abc_rejection_workspace_bytes(chunk))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    counts = (ctypes.c_uint64 * 2)()
    _check(lib.abc_rejection(ctypes.byref(m), _y_obs_host(y_obs), float(eps), m_accept, max_samples,
                             chunk, seed, substream, _ptr(idx), _ptr(rec), counts, _ptr(ws), ws_bytes,
                             _stream(stream)))
    n = int(counts[0])
    return {"idx": idx[:n], "rec": rec[:n], "n_acc": n, "tried": int(counts[1])}


def abc_recalibrate(summ: torch.Tensor, theta: torch.Tensor, acc_idx: torch.Tensor, k: int,
                    stream=None) -> dict:
    """summ [n_obs,n] f64, theta [3,n] f32, acc_idx [q] u32 (CUDA) ->
    {"u": [3,q] f64, "theta_rc": [3,q] f32}."""
    n_obs, n = summ.shape
    q = acc_idx.shape[0]
    dev = summ.device
    u = torch.empty((3, q), dtype=torch.float64, device=dev)
    rc = torch.empty((3, q), dtype=torch.float32, device=dev)
    lib = load_library()
    ws_bytes = int(lib.abc_recalibrate_workspace_bytes(n, k))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    _check(lib.abc_recalibrate(_ptr(summ), _ptr(theta), n, n_obs, _ptr(acc_idx), q, k, _ptr(u), _ptr(rc),
                               _ptr(ws), ws_bytes, _stream(stream)))
    return {"u": u, "theta_rc": rc}


def bege_loglik(theta: torch.Tensor, r: torch.Tensor, h: float, want_logf: bool = False,
                out: dict | None = None, stream=None) -> dict:
    """theta [11, np] f64, r [T] f64 (CUDA) -> {"ll": [np] f64, "logf": [np, T] f64 | None}.
    Pass out={"ll": ..., "ws": ...} to reuse buffers."""
    if theta.dtype != torch.float64 or theta.dim() != 2 or theta.shape[0] != 11:
        raise ValueError("theta must be a [11, np] float64 tensor")
    if r.dtype != torch.float64 or r.dim() != 1:
        raise ValueError("r must be a [T] float64 tensor")
    n_p, T = theta.shape[1], r.shape[0]
    dev = theta.device
    lib = load_library()
    out = dict(out or {})
    ll = out.get("ll")
    if ll is None:
        ll = torch.empty(n_p, dtype=torch.float64, device=dev)
    ws_bytes = int(lib.bege_loglik_workspace_bytes(n_p, T))
    ws = out.get("ws")
    if ws is None or ws.numel() < ws_bytes:
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    logf = torch.empty((n_p, T), dtype=torch.float64, device=dev) if want_logf else None
    _check(lib.bege_loglik(_ptr(theta), n_p, _ptr(r), T, float(h), _ptr(ll), _ptr(logf), _ptr(ws),
                           ws.numel(), _stream(stream)))
    return {"ll": ll, "logf": logf, "ws": ws}


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


def weakinf_test(lambdas: torch.Tensor, lambda0: float, n_obs: int, n_sets: int, alpha: float,
                 seed: int, want_counts: bool = False, stream=None) -> dict:
    """Algorithm 2's alpha-level cut-offs gamma [K] (and counts [K,N] uint32)."""
    K = lambdas.shape[0]
    gamma = torch.empty(K, dtype=torch.float64, device=lambdas.device)
    counts = (torch.empty((K, n_sets), dtype=torch.uint32, device=lambdas.device)
              if want_counts else None)
    lib = load_library()
    ws_bytes = int(lib.weakinf_test_workspace_bytes(K, n_sets))
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=lambdas.device)
    _check(lib.weakinf_test(_ptr(lambdas), K, float(lambda0), n_obs, n_sets, float(alpha), seed,
                            _ptr(gamma), _ptr(counts), _ptr(ws), ws_bytes, _stream(stream)))
    return {"gamma": gamma, "counts": counts}


def toggle_prior_predictive(model: dict, q_obs, n: int, seed: int, substream: int = 0,
                            sample_base: int = 0, want_theta: bool = False, want_summ: bool = False,
                            want_y: bool = False, stream=None) -> dict:
    """Toggle-switch prior predictive: {"theta": [7,n] f32, "summ": [19,n] f64,
    "y": [n,C] f32, "dist": [n] f64} (unrequested outputs are None)."""
    m = ToggleModel.from_dict(model)
    dev = torch.device("cuda")
    q = (ctypes.c_double * 19)(*[float(v) for v in (q_obs.tolist() if hasattr(q_obs, "tolist")
                                                    else q_obs)])
    dist = torch.empty(n, dtype=torch.float64, device=dev)
    theta = torch.empty((7, n), dtype=torch.float32, device=dev) if want_theta else None
    summ = torch.empty((19, n), dtype=torch.float64, device=dev) if want_summ else None
    y = torch.empty((n, m.C), dtype=torch.float32, device=dev) if want_y else None
    _check(load_library().toggle_prior_predictive(ctypes.byref(m), q, n, sample_base, seed, substream,
                                                  _ptr(theta), _ptr(summ), _ptr(y), _ptr(dist),
                                                  _stream(stream)))
    return {"theta": theta, "summ": summ, "y": y, "dist": dist}


# ---------------------------------------------------------------------------
# Batched jobs
# ---------------------------------------------------------------------------

class Batch:
    """A prepared batch of OU-ABC jobs (persistent launch + per-job selection).

    ``jobs`` is a list of dicts with keys model, y_obs, n_samples, seed and
    either k or eps (optionally substream, cap).  Output tensors per job are
    allocated here and returned by :meth:`results`."""

    def __init__(self, jobs: list[dict], tile: tuple[int, int] | None = None, stream=None,
                 device=None):
        self.lib = load_library()
        dev = torch.device(device or "cuda")
        n = len(jobs)
        self.arr = (ABCJob * max(n, 1))()
        self.outs = []
        for j, spec in enumerate(jobs):
            J = self.arr[j]
            J.model = OUModel.from_dict(spec["model"])
            y = [float(v) for v in (spec["y_obs"].tolist() if hasattr(spec["y_obs"], "tolist")
                                    else spec["y_obs"])]
            for i, v in enumerate(y):
                J.y_obs[i] = v
            J.n_samples = int(spec["n_samples"])
            J.seed = int(spec["seed"])
            J.substream = int(spec.get("substream", 0))
            J.k = int(spec.get("k", 0))
            J.eps = float(spec.get("eps", math.inf))
            cap = int(spec.get("cap", J.k if J.k > 0 else J.n_samples))
            o = {"idx": torch.empty(max(cap, 1), dtype=torch.uint32, device=dev),
                 "rec": torch.empty((max(cap, 1), 4), dtype=torch.float32, device=dev),
                 "n_acc": torch.empty(1, dtype=torch.uint64, device=dev),
                 "eps": torch.empty(1, dtype=torch.float64, device=dev),
                 "post": torch.empty(6, dtype=torch.float64, device=dev),
                 "cap": cap}
            if spec.get("keep_dist"):
                o["dist"] = torch.empty(J.n_samples, dtype=torch.float64, device=dev)
                J.dist = o["dist"].data_ptr()
            J.idx_out, J.rec_out, J.cap = o["idx"].data_ptr(), o["rec"].data_ptr(), cap
            J.n_acc_out, J.eps_out, J.post_out = (o["n_acc"].data_ptr(), o["eps"].data_ptr(),
                                                  o["post"].data_ptr())
            self.outs.append(o)
        self.n = n
        ws_bytes = int(self.lib.ppabc_batch_workspace_bytes(self.arr, n))
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.cfg = TileConfig(*(tile or (512, 4096)))
        self.plan = ctypes.c_void_p()
        _check(self.lib.ppabc_batch_prepare(self.arr, n, ctypes.byref(self.cfg), _ptr(self.ws),
                                            ws_bytes, _stream(stream), ctypes.byref(self.plan)))

    def launch(self, graph: bool = False, stream=None) -> None:
        fn = self.lib.ppabc_batch_launch_graph if graph else self.lib.ppabc_batch_launch
        _check(fn(self.plan, _stream(stream)))

    def results(self) -> list[dict]:
        return [{k: (v[:o["cap"]] if k in ("idx", "rec") else v) for k, v in o.items() if k != "cap"}
                for o in self.outs]

    def close(self) -> None:
        if self.plan:
            self.lib.ppabc_batch_plan_destroy(self.plan)
            self.plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Request server
# ---------------------------------------------------------------------------

def abc_request(model: dict, y_obs, n_samples: int, k: int, seed: int, substream: int = 0) -> Request:
    r = Request()
    r.kind = JOB_ABC
    r.substream = substream
    r.seed = seed
    r.model = OUModel.from_dict(model)
    for i, v in enumerate(y_obs.tolist() if hasattr(y_obs, "tolist") else y_obs):
        r.y_obs[i] = float(v)
    r.n_samples = n_samples
    r.k = k
    return r


def pvalue_request(lam: float, n_obs: int, m_sets: int, ybar_obs: float, seed: int) -> Request:
    r = Request()
    r.kind = JOB_PVALUE
    r.seed = seed
    r.lam = lam
    r.n_obs = n_obs
    r.m_sets = m_sets
    r.ybar_obs = ybar_obs
    return r


class Server:
    """Continuous-batching request server over an arena of device memory."""

    def __init__(self, arena_bytes: int, n_slots: int = 8, device=None):
        self.lib = load_library()
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=device or "cuda")
        self.h = ctypes.c_void_p()
        _check(self.lib.ppabc_server_create(_ptr(self.arena), arena_bytes, n_slots,
                                            ctypes.byref(self.h)))

    def submit(self, req: Request) -> int:
        jid = ctypes.c_uint64()
        _check(self.lib.ppabc_server_submit(self.h, ctypes.byref(req), ctypes.byref(jid)))
        return jid.value

    def poll(self, job_id: int) -> dict | None:
        res = Result()
        rc = self.lib.ppabc_server_poll(self.h, job_id, ctypes.byref(res))
        if rc == PPABC_PENDING:
            return None
        _check(rc)
        return res.as_dict()

    def wait(self, job_id: int, timeout_s: float = 60.0) -> dict:
        res = Result()
        _check(self.lib.ppabc_server_wait(self.h, job_id, timeout_s, ctypes.byref(res)))
        return res.as_dict()

    def fetch(self, job_id: int, cap: int):
        import numpy as np
        idx = np.zeros(max(cap, 1), dtype=np.uint32)
        rec = np.zeros((max(cap, 1), 4), dtype=np.float32)
        n = ctypes.c_uint64()
        _check(self.lib.ppabc_server_fetch(self.h, job_id, idx.ctypes.data_as(ctypes.c_void_p),
                                           rec.ctypes.data_as(ctypes.c_void_p), cap,
                                           ctypes.byref(n)))
        return idx[:n.value], rec[:n.value]

    def release(self, job_id: int) -> None:
        _check(self.lib.ppabc_server_release(self.h, job_id))

    def cancel(self, job_id: int) -> None:
        _check(self.lib.ppabc_server_cancel(self.h, job_id))

    def stats(self) -> dict:
        st = ServerStats()
        _check(self.lib.ppabc_server_get_stats(self.h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def now(self) -> float:
        return float(self.lib.ppabc_server_now(self.h))

    def close(self) -> None:
        if self.h:
            self.lib.ppabc_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
