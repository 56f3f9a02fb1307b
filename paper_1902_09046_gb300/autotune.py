"""Tile autotuner for the persistent batched kernel.

The persistent kernel's tile shape -- CTA width and the least number of
Euler-Maruyama steps a thread runs per tile -- trades scheduling overhead (an
atomic per tile) against load balance at the end of the launch.  The tuner
times each candidate on a scaled-down copy of the job mix (same step counts,
fewer samples per job) with CUDA events and keeps the fastest.  Results are
cached per (GPU name, step-count profile) in a JSON file so a mix is tuned
once per machine.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import binding

CANDIDATES = ((512, 1024), (512, 4096), (512, 16384), (256, 4096))


def _cache_path() -> str:
    root = os.environ.get("PPABC_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache",
                                                             "ppabc_gb300")
    return os.path.join(root, "autotune.json")


def _profile_key(jobs: list[dict]) -> str:
    steps = np.array([j["model"]["n_steps"] for j in jobs], dtype=np.float64)
    sizes = np.array([j["n_samples"] for j in jobs], dtype=np.float64)
    hist_s = np.histogram(np.log2(steps), bins=8, range=(0, 16))[0]
    hist_n = np.histogram(np.log2(sizes), bins=8, range=(0, 32))[0]
    digest = hashlib.sha1((hist_s.tobytes() + hist_n.tobytes())).hexdigest()[:12]
    return f"{torch.cuda.get_device_name()}|{len(jobs)}|{digest}"


def _scaled(jobs: list[dict], max_samples: int) -> list[dict]:
    out = []
    for j in jobs:
        n = int(min(j["n_samples"], max_samples))
        k = j.get("k", 0)
        spec = dict(j, n_samples=n)
        if k:
            spec["k"] = max(1, min(n, int(round(k * n / j["n_samples"]))))
        spec.pop("keep_dist", None)
        out.append(spec)
    return out


def time_config(jobs: list[dict], tile: tuple[int, int], reps: int = 2) -> float:
    b = binding.Batch(jobs, tile=tile)
    try:
        b.launch()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            ev0.record()
            b.launch()
            ev1.record()
            ev1.synchronize()
            best = min(best, ev0.elapsed_time(ev1))
        return best
    finally:
        b.close()


def tune(jobs: list[dict], candidates=CANDIDATES, max_samples: int = 200_000,
         use_cache: bool = True) -> tuple[int, int]:
    """Best (threads, min_tile_steps) for this job mix on the current GPU."""
    key = _profile_key(jobs)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return tuple(cache[key]["tile"])
    probe = _scaled(jobs, max_samples)
    times = {tile: time_config(probe, tile) for tile in candidates}
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"tile": list(best), "ms": {f"{t[0]}x{t[1]}": v for t, v in times.items()}}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return best
