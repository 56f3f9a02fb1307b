"""Sharding over ranks (CPU, gloo, world size 2): per-rank oracle shards plus
the merge give exactly the unsharded accepted set and tail counts."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1902_09046_gb300 import shard, workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, k, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workloads.abc_small()
    model = dict(w.model, n_steps=200, dt=10.0 / 200)
    base, cnt = shard.shard_range(rank, world, n)
    _, _, d = oracle.ou_prior_predictive(model, w.y_obs, cnt, seed=w.seed, base=base, n_threads=2)
    loc = oracle.select_topk(d, min(k, cnt)).astype(np.int64)
    idx, eps = shard.gather_topk(d[loc], loc + base, k)
    pv = workloads.pvalue_sweep_workload(m_sets=4000)
    mb, mc = shard.shard_range(rank, world, pv.m_sets)
    c, _, _ = oracle.pvalue_sweep(pv.lambdas[:8], pv.n_obs, mc, pv.ybar_obs, pv.seed, base=mb,
                                  n_threads=2)
    total = shard.allreduce_counts(c)
    q.put((rank, idx.tolist(), float(eps), total.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shard_merge_equals_unsharded():
    n, k, world = 3000, 37, 2
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
    _, _, d = oracle.ou_prior_predictive(model, w.y_obs, n, seed=w.seed)
    ref = oracle.select_topk(d, k).astype(np.int64).tolist()
    pv = workloads.pvalue_sweep_workload(m_sets=4000)
    c_ref, _, _ = oracle.pvalue_sweep(pv.lambdas[:8], pv.n_obs, pv.m_sets, pv.ybar_obs, pv.seed)
    for rank, idx, eps, total in res:
        assert idx == ref
        assert eps == np.sort(d)[k - 1]
        assert total == c_ref.tolist()


def test_merge_topk_ties_and_nan():
    idx, eps = shard.merge_topk([np.array([1.0, np.nan]), np.array([1.0, 0.5])],
                                [np.array([10, 11]), np.array([3, 4])], 3)
    np.testing.assert_array_equal(idx, [3, 4, 10])
    assert eps == 1.0
    with pytest.raises(ValueError):
        shard.merge_topk([np.array([1.0])], [np.array([0])], 2)


def test_shard_range_covers_everything():
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            got = [shard.shard_range(r, world, n) for r in range(world)]
            assert sum(c for _, c in got) == n
            assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))
