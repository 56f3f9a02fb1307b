"""Sharding over ranks (CPU, gloo, world size 2): each rank computes its
oracle shard, builds its candidate record and calls shard.merge_topk and
shard.allreduce_counts -- the functions bench.py --gpus N calls over NCCL --
with the oracle's selection in place of the device kernel.  The merged
accepted set, epsilon, posterior moments and tail counts equal the unsharded
ones exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1902_09046_gb300 import shard, workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def oracle_merge(d, index, theta, k):
    """The merge selection done by the oracle on host tensors (what the device
    kernel abc_merge_candidates computes)."""
    pos = oracle.select_topk(d.numpy(), k).astype(np.int64)
    th = theta.numpy().T.astype(np.float64)
    mean, var = oracle.moments(th, pos.astype(np.uint64))
    return {"idx": torch.from_numpy(index.numpy()[pos]), "eps": float(d.numpy()[pos].max()),
            "post": np.concatenate([mean, var])}


def _worker(rank, world, port, n, k, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workloads.abc_small()
    model = dict(w.model, n_steps=200, dt=10.0 / 200)
    # uneven ranges (world does not divide n) and ranks with fewer samples than k
    base, cnt = shard.shard_range(rank, world, n)
    th, _, d = oracle.ou_prior_predictive(model, w.y_obs, cnt, seed=w.seed, base=base, n_threads=2)
    loc = oracle.select_topk(d, min(k, cnt)).astype(np.int64)
    cand = {"dist": torch.from_numpy(d[loc].copy()),
            "index": torch.from_numpy((loc + base).astype(np.uint64)),
            "theta": torch.from_numpy(th[loc].T.astype(np.float32).copy())}
    res = shard.merge_topk(cand, k, merge=oracle_merge)
    pv = workloads.pvalue_sweep_workload(m_sets=4000)
    mb, mc = shard.shard_range(rank, world, pv.m_sets)
    c, _, _ = oracle.pvalue_sweep(pv.lambdas[:8], pv.n_obs, mc, pv.ybar_obs, pv.seed, base=mb,
                                  n_threads=2)
    total = shard.allreduce_counts(torch.from_numpy(c.astype(np.uint64)), max_count_per_rank=mc)
    q.put((rank, res["idx"].numpy().astype(np.int64).tolist(), res["eps"], res["post"].tolist(),
           total.numpy().astype(np.uint64).tolist(), str(total.dtype)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n,k", [(3000, 37), (41, 30)])
def test_two_rank_shard_merge_equals_unsharded(n, k):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, k, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = workloads.abc_small()
    model = dict(w.model, n_steps=200, dt=10.0 / 200)
    th, _, d = oracle.ou_prior_predictive(model, w.y_obs, n, seed=w.seed)
    ref = oracle.select_topk(d, k).astype(np.int64)
    mean, var = oracle.moments(th.astype(np.float32).astype(np.float64), ref.astype(np.uint64))
    pv = workloads.pvalue_sweep_workload(m_sets=4000)
    c_ref, _, _ = oracle.pvalue_sweep(pv.lambdas[:8], pv.n_obs, pv.m_sets, pv.ybar_obs, pv.seed)
    for rank, idx, eps, post, total, dtype in res:
        assert idx == ref.tolist()
        assert eps == np.sort(d)[k - 1]
        np.testing.assert_array_equal(post, np.concatenate([mean, var]))
        assert total == c_ref.tolist()
        assert dtype == "torch.uint64"


def test_allreduce_counts_guards_the_int64_range():
    with pytest.raises(ValueError):
        shard.allreduce_counts(torch.zeros(3, dtype=torch.int64), 1)


def test_shard_range_covers_everything():
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            got = [shard.shard_range(r, world, n) for r in range(world)]
            assert sum(c for _, c in got) == n
            assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))
