"""Batched persistent execution: every job's results are bit-identical to the
job run alone (abc_prior_predictive + abc_select), for any tile shape, eager
or graph-replayed; a small job is checked against the oracle."""
import math

import numpy as np
import pytest

import oracle
from gpu_common import BAND, band_check, require_gpu, to_np, torch
from paper_1902_09046_gb300 import workloads

pytestmark = pytest.mark.gpu


def _mix():
    rng = np.random.default_rng(11)
    jobs = []
    for j, (n, s) in enumerate([(1000, 100), (50_000, 37), (12_345, 1000), (129, 4),
                                (70_001, 250), (3, 10), (20_000, 2000), (4096, 100)]):
        theta = tuple(float(rng.uniform(lo, hi)) for lo, hi in
                      zip(workloads.OU_PRIOR_LO, workloads.OU_PRIOR_HI))
        t_end = 0.4 if s < 10 else 10.0
        spec = {"model": workloads.ou_model(s, t_end=t_end, n_obs=min(10, s)),
                "y_obs": workloads.ou_observed(theta, seed=100 + j, t_end=t_end, n_obs=min(10, s)),
                "n_samples": n, "seed": 1000 + j, "substream": j % 3}
        if j % 3 == 2:
            spec["eps"] = 1.0
            spec["cap"] = n
        else:
            spec["k"] = max(1, n // 100)
        jobs.append(spec)
    return jobs


def _alone(binding, spec):
    out = binding.abc_prior_predictive(spec["model"], spec["y_obs"], spec["n_samples"], spec["seed"],
                                       substream=spec["substream"], want_theta=False)
    k = spec.get("k", 0)
    sel = binding.abc_select(out["dist"], k=k, eps=spec.get("eps", math.inf), model=spec["model"],
                             seed=spec["seed"], substream=spec["substream"], cap=spec.get("cap"))
    return out["dist"], sel


def _same(a, b):
    n = int(to_np(a["n_acc"])[0])
    assert n == int(to_np(b["n_acc"])[0])
    w = min(n, a["idx"].shape[0])
    np.testing.assert_array_equal(to_np(a["idx"][:w]), to_np(b["idx"][:w]))
    np.testing.assert_array_equal(to_np(a["rec"][:w]), to_np(b["rec"][:w]))
    np.testing.assert_array_equal(to_np(a["eps"]), to_np(b["eps"]))
    np.testing.assert_array_equal(to_np(a["post"]), to_np(b["post"]))


@pytest.mark.parametrize("tile", [(512, 4096), (256, 1024), (512, 1)])
def test_batched_equals_alone(tile):
    binding = require_gpu()
    jobs = _mix()
    for spec in jobs:
        spec["keep_dist"] = True
    b = binding.Batch(jobs, tile=tile)
    b.launch()
    torch.cuda.synchronize()
    res = b.results()
    for spec, r in zip(jobs, res):
        d, sel = _alone(binding, spec)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_np(r["dist"]), to_np(d))
        _same(r, sel)
    b.close()


def test_graph_replay_is_identical():
    binding = require_gpu()
    jobs = _mix()
    b = binding.Batch(jobs, tile=(512, 4096))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.launch(graph=True, stream=s)
        s.synchronize()
        first = [{k: v.clone() for k, v in r.items()} for r in b.results()]
        for r in b.results():
            r["n_acc"].zero_()
        b.launch(graph=True, stream=s)
        s.synchronize()
    for a, r in zip(first, b.results()):
        _same(a, r)
    b.close()


def test_batched_job_matches_oracle():
    binding = require_gpu()
    w = workloads.abc_small()
    spec = {"model": w.model, "y_obs": w.y_obs, "n_samples": 5000, "seed": w.seed, "k": 50,
            "keep_dist": True}
    other = dict(spec, seed=77, n_samples=30_000, k=300, keep_dist=False)
    b = binding.Batch([other, spec])
    b.launch()
    torch.cuda.synchronize()
    r = b.results()[1]
    _, _, d_o = oracle.ou_prior_predictive(w.model, w.y_obs, 5000, seed=w.seed)
    np.testing.assert_allclose(to_np(r["dist"]), d_o, rtol=1e-5)
    idx_o = oracle.select_topk(d_o, 50)
    band_check(to_np(r["idx"]), idx_o, d_o, np.sort(d_o)[49], BAND)
    b.close()


def test_invalid_job_is_rejected():
    binding = require_gpu()
    jobs = _mix()
    jobs[3]["k"] = jobs[3]["n_samples"] + 1
    with pytest.raises(binding.PPABCError):
        binding.Batch(jobs)
