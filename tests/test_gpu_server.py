"""Request server: results are identical alone and in a concurrent mix;
admission by device footprint; cancellation and host-side timeouts (no GPU
fault is involved in any failure test)."""
import math
import time

import numpy as np
import pytest

from gpu_common import require_gpu, to_np, torch
from paper_1902_09046_gb300 import workloads

pytestmark = pytest.mark.gpu


def _alone_abc(binding, model, y, n, k, seed):
    out = binding.abc_prior_predictive(model, y, n, seed, want_theta=False)
    sel = binding.abc_select(out["dist"], k=k, model=model, seed=seed)
    torch.cuda.synchronize()
    return sel


def _alone_pv(binding, lam, n_obs, m, ybar, seed):
    lt = torch.tensor([lam], dtype=torch.float64, device="cuda")
    out = binding.pvalue_sweep(lt, n_obs, m, ybar, seed)
    torch.cuda.synchronize()
    return int(to_np(out["counts"])[0]), float(to_np(out["p"])[0])


def _jobs():
    jobs = workloads.served_jobs(rate_per_s=200, duration_s=0.2, gen_seed=4)
    return jobs[:24]


def _request(binding, j):
    if j.kind == "abc":
        return binding.abc_request(j.model, j.y_obs, j.n, j.k_accept, j.seed)
    return binding.pvalue_request(j.lam, j.n_obs, j.n, j.ybar_obs, j.seed)


@pytest.mark.parametrize("slots", [1, 6])
def test_results_identical_alone_and_in_the_mix(slots):
    binding = require_gpu()
    jobs = _jobs()
    assert {j.kind for j in jobs} == {"abc", "pvalue"}
    with binding.Server(1 << 30, n_slots=slots) as srv:
        ids = [srv.submit(_request(binding, j)) for j in jobs]
        res = [srv.wait(i, 120.0) for i in ids]
        for j, jid, r in zip(jobs, ids, res):
            assert r["status"] == binding.PPABC_OK
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
            if j.kind == "abc":
                ref = _alone_abc(binding, j.model, j.y_obs, j.n, j.k_accept, j.seed)
                assert r["n_acc"] == int(to_np(ref["n_acc"])[0]) == j.k_accept
                assert r["eps"] == float(to_np(ref["eps"])[0])
                np.testing.assert_array_equal(np.array(r["post"]), to_np(ref["post"]))
                idx, rec = srv.fetch(jid, j.k_accept)
                np.testing.assert_array_equal(idx, to_np(ref["idx"]))
                np.testing.assert_array_equal(rec, to_np(ref["rec"]))
                assert (r["count"], r["p"]) == (0, 0.0)  # p-value fields untouched
            else:
                c, p = _alone_pv(binding, j.lam, j.n_obs, j.n, j.ybar_obs, j.seed)
                assert (r["count"], r["p"]) == (c, p)
                assert (r["n_acc"], r["eps"]) == (0, 0.0)  # ABC fields untouched
            srv.release(jid)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert st["arena_used_bytes"] == 0


def test_admission_by_device_footprint():
    binding = require_gpu()
    w = workloads.abc_small()
    with binding.Server(4 << 20, n_slots=4) as srv:  # 4 MiB arena
        with pytest.raises(binding.PPABCError) as e:
            srv.submit(binding.abc_request(w.model, w.y_obs, 1_000_000, 100, 1))  # 8 MB of distances
        assert e.value.code == binding.PPABC_ENOMEM
        # jobs of ~1.7 MiB each: at most two fit at a time, all complete
        ids = [srv.submit(binding.abc_request(w.model, w.y_obs, 200_000, 50, s)) for s in range(6)]
        for i in ids:
            assert srv.wait(i, 60.0)["status"] == binding.PPABC_OK
            srv.release(i)
        assert srv.stats()["peak_arena_bytes"] <= 4 << 20


def test_cancel_and_timeout_are_host_side():
    binding = require_gpu()
    w = workloads.abc_small()
    big = dict(w.model, n_steps=20_000, dt=10.0 / 20_000)
    with binding.Server(1 << 30, n_slots=1) as srv:
        first = srv.submit(binding.abc_request(big, w.y_obs, 2_000_000, 100, 1))
        queued = [srv.submit(binding.abc_request(w.model, w.y_obs, 1000, 10, s)) for s in range(3)]
        srv.cancel(queued[1])
        with pytest.raises(binding.PPABCError) as e:
            srv.wait(first, 1e-4)  # still running: the host wait gives up, the GPU is untouched
        assert e.value.code == binding.PPABC_ETIMEOUT
        assert srv.wait(first, 120.0)["status"] == binding.PPABC_OK
        assert srv.wait(queued[1], 60.0)["status"] == binding.PPABC_ECANCELLED
        for i in (queued[0], queued[2]):
            assert srv.wait(i, 60.0)["status"] == binding.PPABC_OK
        with pytest.raises(binding.PPABCError):
            srv.fetch(queued[1], 10)
        with pytest.raises(binding.PPABCError):
            srv.submit(binding.abc_request(w.model, w.y_obs, 10, 11, 1))  # k > n
