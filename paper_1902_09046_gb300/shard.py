"""Sharding of the prior-predictive path over ranks (host side).

Samples are independent and every random number is keyed by the global
sample (or data-set) index, so a job splits into contiguous index ranges, one
per rank, with no communication while simulating.  The only exchange is the
final merge:
  * ABC: each rank keeps its local k nearest; the global k nearest by
    (distance, index) are among the P*k candidates, so one small gather and
    a host-side selection give exactly the unsharded accepted set;
  * p-value: tail counts of disjoint data-set ranges add up.
"""
from __future__ import annotations

import numpy as np


def shard_range(rank: int, world: int, n: int) -> tuple[int, int]:
    """Contiguous (base, count) of rank among world ranks covering 0..n-1."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi - lo


def merge_topk(dists: list[np.ndarray], indices: list[np.ndarray], k: int):
    """Global k nearest from per-rank candidates (distance, global index).

    Ties go to the smaller index and NaN sorts last, as in the single-rank
    selection.  Returns (indices ascending, the k-th smallest distance)."""
    d = np.concatenate([np.asarray(x, dtype=np.float64) for x in dists])
    i = np.concatenate([np.asarray(x, dtype=np.int64) for x in indices])
    if k > d.size:
        raise ValueError("fewer candidates than k")
    nan = np.isnan(d)
    order = np.lexsort((i, d, nan))  # NaN last, then distance, then index
    take = order[:k]
    eps = d[take[-1]] if k > 0 else np.nan
    return np.sort(i[take]), eps


def merge_counts(counts: list[np.ndarray]) -> np.ndarray:
    """Sum of per-rank uint64 tail counts."""
    out = np.zeros_like(np.asarray(counts[0], dtype=np.uint64))
    for c in counts:
        out += np.asarray(c, dtype=np.uint64)
    return out


def gather_topk(dist_local: np.ndarray, idx_global: np.ndarray, k: int, group=None):
    """All-gathers per-rank candidates with torch.distributed and merges them
    on every rank (the candidate lists are k entries per rank)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    pay = torch.from_numpy(np.stack([np.asarray(dist_local, dtype=np.float64),
                                     np.asarray(idx_global, dtype=np.float64)]))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([pay.shape[1]], dtype=torch.int64), group=group)
    m = int(max(s.item() for s in sizes))
    padded = torch.full((2, m), float("nan"), dtype=torch.float64)
    padded[:, :pay.shape[1]] = pay
    bufs = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(bufs, padded, group=group)
    ds, ix = [], []
    for s, b in zip(sizes, bufs):
        n = int(s.item())
        ds.append(b[0, :n].numpy())
        ix.append(b[1, :n].numpy().astype(np.int64))
    return merge_topk(ds, ix, k)


def allreduce_counts(counts: np.ndarray, group=None) -> np.ndarray:
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.asarray(counts, dtype=np.int64).copy())
    dist.all_reduce(t, group=group)
    return t.numpy().astype(np.uint64)
