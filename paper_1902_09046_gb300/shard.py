"""Sharding of the prior-predictive path over ranks.

Samples are independent and every random number is keyed by the global
sample (or data-set) index, so a job splits into contiguous index ranges, one
per rank (the static split of the paper's sampler, Sec. 3.4), with no
communication while simulating.  The only exchange is the final merge:

  * ABC (the fixed-N selection of Sec. 3.1): each rank selects its own k
    nearest with abc_select and turns them into a candidate record
    (abc_select_candidates: binary64 distance, global index, theta); the
    records are all-gathered in rank order, which for contiguous ranges is
    ascending global index, and abc_merge_candidates selects the global k
    nearest with the same kernels -- exactly the unsharded accepted set,
    epsilon and posterior moments;
  * p-value (Sec. 4.1): the exact tail counts of disjoint data-set ranges
    add up (an all-reduce of 64-bit integers).

The collectives are torch.distributed (NCCL between GPUs, gloo on the host);
the selection itself runs in the library's kernels.
"""
from __future__ import annotations

import torch

INT64_MAX = (1 << 63) - 1


def shard_range(rank: int, world: int, n: int) -> tuple[int, int]:
    """Contiguous (base, count) of rank among world ranks covering 0..n-1."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi - lo


def gather_candidates(cand: dict, group=None) -> dict:
    """All-gathers every rank's candidate record {"dist": [c] f64, "index":
    [c] u64, "theta": [3,c] f32} (tensors on the collective's device: CUDA for
    NCCL, CPU for gloo) and concatenates them in rank order.  Records may
    differ in length; they travel padded to the longest.  The global indices
    travel as the same 64 bits viewed as int64 (no conversion)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    d, ix, th = cand["dist"], cand["index"], cand["theta"]
    dev = d.device
    c = d.shape[0]
    n = torch.tensor([c], dtype=torch.int64, device=dev)
    sizes = [torch.empty_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    pd = torch.full((m,), float("inf"), dtype=torch.float64, device=dev)
    pi = torch.zeros(m, dtype=torch.int64, device=dev)
    pt = torch.zeros((3, m), dtype=torch.float32, device=dev)
    pd[:c] = d
    pi[:c] = ix.view(torch.int64)
    pt[:, :c] = th
    bd = [torch.empty_like(pd) for _ in range(world)]
    bi = [torch.empty_like(pi) for _ in range(world)]
    bt = [torch.empty_like(pt) for _ in range(world)]
    dist.all_gather(bd, pd, group=group)
    dist.all_gather(bi, pi, group=group)
    dist.all_gather(bt, pt.contiguous(), group=group)
    return {"dist": torch.cat([b[:s] for b, s in zip(bd, sizes)]),
            "index": torch.cat([b[:s] for b, s in zip(bi, sizes)]).view(torch.uint64),
            "theta": torch.cat([b[:, :s] for b, s in zip(bt, sizes)], dim=1).contiguous()}


def merge_topk(cand: dict, k: int, group=None, merge=None) -> dict:
    """Global k nearest of a sample-sharded job from this rank's candidate
    record: gathers the records of all ranks and selects with `merge`
    (default: the library's abc_merge_candidates, on the device).  Returns
    {"idx": [k] global indices, "rec", "n_acc", "eps", "post"} on every rank."""
    allc = gather_candidates(cand, group)
    if merge is None:
        from . import binding
        merge = binding.abc_merge_candidates
    if allc["dist"].shape[0] < k:
        raise ValueError("fewer candidates than k")
    return merge(allc["dist"], allc["index"], allc["theta"], k)


def allreduce_counts(counts: torch.Tensor, max_count_per_rank: int, group=None) -> torch.Tensor:
    """Exact sum over ranks of uint64 tail counts of disjoint data-set ranges.
    The all-reduce adds the same bits as int64, which is exact while every
    partial sum stays below 2^63: asserted from the per-rank bound (the
    number of data sets a rank draws per lambda)."""
    import torch.distributed as dist

    if counts.dtype != torch.uint64:
        raise ValueError("counts must be uint64")
    world = dist.get_world_size(group)
    if max_count_per_rank * world > INT64_MAX:
        raise OverflowError("the summed counts could exceed 2^63")
    t = counts.clone().view(torch.int64)
    dist.all_reduce(t, group=group)
    return t.view(torch.uint64)
