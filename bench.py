#!/usr/bin/env python3
"""Benchmark of the prior-predictive hot path on GB300.

One step is one pass of the whole path over one batch of synthetic input:
  * OU-ABC, N = 2^24 prior samples x 10^4 Euler-Maruyama steps (dt = 1e-3),
    10 observations, accept the 0.1% nearest (k = 16777) with posterior
    moments: abc_prior_predictive + abc_select;
  * p-value sweep, 64 lambdas x 10^6 data sets x (n = 50) + 1 normals:
    pvalue_sweep.
The metric is path-steps per second (an EM step of one sample, or one normal
of one p-value data set), whole job, inputs resident in HBM.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores over a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1902_09046_gb300 import workloads  # noqa: E402

METRIC = "EM path-steps/sec (+ frac of FP32/MUFU roofline)"
UNIT = "path-steps/s"
MUFU_PER_SM_CLK = 16          # special-function (MUFU) lanes per SM per clock
MUFU_PER_PATH_STEP = 2.0      # log, sqrt, sin, cos per Box-Muller pair = 2 per normal
KERNEL_SOURCES = ("paper_1902_09046_gb300/csrc/em_ou.cu", "paper_1902_09046_gb300/csrc/ou_path.cuh",
                  "paper_1902_09046_gb300/csrc/rng.cuh", "paper_1902_09046_gb300/csrc/bm_table.cuh",
                  "paper_1902_09046_gb300/csrc/bm_tables.h")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--mode", choices=("path", "batch", "serve", "toggle", "configs", "bege"), default="path",
                    help="path: the headline step; batch: 256 uneven jobs, plain vs persistent; "
                         "serve: Poisson arrivals, served vs plain")
    ap.add_argument("--jobs", type=int, default=256)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--abc-samples", type=int, default=1 << 24)
    ap.add_argument("--abc-steps", type=int, default=10_000)
    ap.add_argument("--pv-sets", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-latency", action="store_true",
                    help="skip the batched-vs-plain and served-vs-plain blocks of the default run")
    ap.add_argument("--batch-repeats", type=int, default=10)
    ap.add_argument("--latency-serve-seconds", type=float, default=10.0,
                    help="length of the served-vs-plain replay in the default run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_config(args):
    abc = workloads.abc_large(args.abc_samples)
    abc.model = workloads.ou_model(args.abc_steps)
    abc.k_accept = max(1, int(0.001 * args.abc_samples))
    pv = workloads.pvalue_sweep_workload(args.pv_sets)
    return abc, pv


def path_steps_per_step(abc, pv):
    abc_steps = abc.n_samples * abc.model["n_steps"]
    pv_steps = len(pv.lambdas) * pv.m_sets * (pv.n_obs + 1)
    return abc_steps, pv_steps


def config_dict(abc, pv, world, k_accept=None):
    k = abc.k_accept if k_accept is None else k_accept
    return {
        "workload": (f"ou_abc N={abc.n_samples} S={abc.model['n_steps']} dt={abc.model['dt']:g} "
                     f"k={k} + pvalue K={len(pv.lambdas)} M={pv.m_sets} n={pv.n_obs}"),
        "abc_samples_per_rank": abc.n_samples, "em_steps": abc.model["n_steps"],
        "k_accept": k, "pvalue_lambdas": len(pv.lambdas), "pvalue_sets": pv.m_sets,
        "pvalue_n": pv.n_obs, "sharding": f"sample and data-set ranges over {world} rank(s)",
        "l2": "flushed between timed steps (256 MiB write)",
    }


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline leg only)
# ---------------------------------------------------------------------------

def run_oracle_sample(abc, pv, frac, threads):
    """Runs the oracle on the first `frac` of the ABC samples and of the
    p-value data sets; returns (path_steps, seconds)."""
    import oracle
    n_abc = max(1, int(round(abc.n_samples * frac)))
    m_pv = max(1, int(round(pv.m_sets * frac)))
    t0 = time.perf_counter()
    _, _, dist = oracle.ou_prior_predictive(abc.model, abc.y_obs, n_abc, seed=abc.seed,
                                            want_theta=True, n_threads=threads)
    k = max(1, int(0.001 * n_abc))
    idx = oracle.select_topk(dist, k)
    oracle.pvalue_sweep(pv.lambdas, pv.n_obs, m_pv, pv.ybar_obs, pv.seed, n_threads=threads)
    dt = time.perf_counter() - t0
    steps = n_abc * abc.model["n_steps"] + len(pv.lambdas) * m_pv * (pv.n_obs + 1)
    del idx
    return steps, dt


def calibrate_fraction(abc, pv, threads, target_s):
    frac = 2048.0 / abc.n_samples
    steps, dt = run_oracle_sample(abc, pv, frac, threads)
    while dt < 0.5 and frac < 1.0:
        frac = min(1.0, frac * 4)
        steps, dt = run_oracle_sample(abc, pv, frac, threads)
    return min(1.0, frac * target_s / max(dt, 1e-6))


def cpu_baseline(abc, pv, target_s):
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    frac = calibrate_fraction(abc, pv, threads, target_s)
    steps, dt = run_oracle_sample(abc, pv, frac, threads)
    # The same oracle on one core, on a sample 1/threads the size (about the
    # same wall time).
    frac1 = frac / threads
    steps1, dt1 = run_oracle_sample(abc, pv, frac1, 1)
    return {"value": steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"first {frac:.3g} of the workload: {int(round(abc.n_samples * frac))} ABC samples "
                       f"x {abc.model['n_steps']} steps + {len(pv.lambdas)} x {int(round(pv.m_sets * frac))} "
                       f"p-value data sets; FP64, static split over {threads} threads; {dt:.1f} s"),
            "single_core": {"value": steps1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"first {frac1:.3g} of the workload on one thread; {dt1:.1f} s"}}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    abc, pv = workload_config(args)
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    frac = calibrate_fraction(abc, pv, threads, 4.0)
    for _ in range(args.warmup):
        run_oracle_sample(abc, pv, frac, threads)
    total_steps, total_s, per = 0, 0.0, []
    for _ in range(args.steps):
        s, dt = run_oracle_sample(abc, pv, frac, threads)
        total_steps += s
        total_s += dt
        per.append(dt)
    value = total_steps / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": config_dict(abc, pv, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step: first {frac:.3g} of the workload on the host cores"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(n_samples):
    """DRAM bytes per em_ou_fused_x2 launch from the committed ncu summary, scaled
    to this launch size; None if absent or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "em_ou_fused_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash() or rec.get("dram_bytes") is None:
        return None
    return float(rec["dram_bytes"]) * n_samples / float(rec["n_samples"])


def device_props(binding):
    """SM count and maximum SM clock of the current device, read at run time
    (the roofline and the pipe ceilings are built from them)."""
    sms, mhz = binding.device_info()
    return {"sm_count": int(sms), "sm_max_mhz": float(mhz)}


def pipe_bounds(ms_per_launch, path_steps, dev):
    """The per-pipe ceilings of the kernel from its measured cycles per warp
    step (32 path-steps) on one SM sub-partition -- issue slots, ALU-pipe
    cycles, FMA-pipe cycles, cycles of its heavy sub-pipe -- read from the
    committed ncu summary; None if
    absent or the kernel changed since.  Each ceiling is the path-step rate if
    that resource alone were busy all the time."""
    path = os.path.join(ROOT, "profiles", "em_ou_fused_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    cyc = rec.get("smsp_cycles_per_warp_step")
    if not cyc or rec.get("source_hash") != kernel_source_hash():
        return None
    achieved = path_steps / (ms_per_launch / 1e3)
    smsp_cycles_per_s = dev["sm_count"] * 4 * dev["sm_max_mhz"] * 1e6
    out = {"cycles_per_warp_step": cyc}
    for name, c in cyc.items():
        if name == "elapsed":
            continue
        ceiling = smsp_cycles_per_s * 32 / c
        out[name] = {"ceiling_path_steps_per_s": ceiling, "frac": achieved / ceiling}
    binding = min((k for k in out if k != "cycles_per_warp_step"),
                  key=lambda k: out[k]["ceiling_path_steps_per_s"])
    out["binding"] = binding
    return out


def gpu_arm(args):
    import torch
    from paper_1902_09046_gb300 import binding
    from paper_1902_09046_gb300 import build as libbuild

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    libbuild.build()
    binding.device_check()
    dev_props = device_props(binding)
    abc, pv = workload_config(args)
    N = abc.n_samples
    base = rank * N
    if base + N > (1 << 32):
        raise SystemExit("sample range of this rank exceeds 2^32")
    set_base = rank * pv.m_sets  # each rank draws its own p-value data sets
    if set_base + pv.m_sets > (1 << 32):
        raise SystemExit("p-value data-set range of this rank exceeds 2^32")
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    lam_host = torch.tensor(pv.lambdas, dtype=torch.float64).pin_memory()
    lam_dev = lam_host.to(dev)
    dist_buf = torch.empty(N, dtype=torch.float64, device=dev)
    ws = torch.empty(binding.abc_select_workspace_bytes(N), dtype=torch.uint8, device=dev)
    # One job of N x world samples: each rank keeps its own k nearest of the
    # global k (k_local = min(k, N)); with world > 1 the ranks then merge
    # their candidates (shard.merge_topk over NCCL) into the global accepted
    # set, and all-reduce the p-value tail counts.
    k_global = max(1, int(0.001 * N * world))
    k_local = min(k_global, N)
    sel_out = {"idx": torch.empty(k_local, dtype=torch.uint32, device=dev),
               "rec": torch.empty((k_local, 4), dtype=torch.float32, device=dev),
               "n_acc": torch.empty(1, dtype=torch.uint64, device=dev),
               "eps": torch.empty(1, dtype=torch.float64, device=dev),
               "post": torch.empty(6, dtype=torch.float64, device=dev)}
    pv_out = {"counts": torch.empty(len(pv.lambdas), dtype=torch.uint64, device=dev),
              "p": torch.empty(len(pv.lambdas), dtype=torch.float64, device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    launches_per_step = 1 + 11 + 2 + (2 + 12 if world > 1 else 0)
    merged = {}

    def step(em_events=None):
        if em_events is not None:
            em_events[0].record(stream)
        binding.abc_prior_predictive(abc.model, abc.y_obs, N, abc.seed, sample_base=base,
                                     want_theta=False, out={"dist": dist_buf}, stream=stream)
        if em_events is not None:
            em_events[1].record(stream)
        binding.abc_select(dist_buf, k=k_local, model=abc.model, seed=abc.seed, sample_base=base,
                           workspace=ws, out=sel_out, stream=stream)
        binding.pvalue_sweep(lam_dev, pv.n_obs, pv.m_sets, pv.ybar_obs, pv.seed, set_base=set_base,
                             out=pv_out, stream=stream)
        if world > 1:
            from paper_1902_09046_gb300 import shard
            cand = binding.abc_select_candidates(dist_buf, sel_out, k_local, sample_base=base, stream=stream)
            merged.update(shard.merge_topk(cand, k_global))
            merged["counts"] = shard.allreduce_counts(pv_out["counts"], pv.m_sets)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    steps_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
    em_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    with ClockSampler(local_rank) as clocks:
        barrier()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)  # L2 flush between timed steps, outside the step events
            steps_ev[i][0].record(stream)
            step(em_ev[i])
            steps_ev[i][1].record(stream)
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in steps_ev]
    em_ms = [a.elapsed_time(b) for a, b in em_ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    abc_steps, pv_steps = path_steps_per_step(abc, pv)
    units = (abc_steps + pv_steps) * world * args.steps
    value = units / (total_ms / 1e3)

    # End to end through the public API with host buffers: H2D of the step's
    # inputs (lambda grid; the OU model and observed data travel as launch
    # arguments) and D2H of every result, inside the timed region.
    host_out = {"idx": torch.empty(abc.k_accept, dtype=torch.uint32).pin_memory(),
                "rec": torch.empty((abc.k_accept, 4), dtype=torch.float32).pin_memory(),
                "n_acc": torch.empty(1, dtype=torch.uint64).pin_memory(),
                "eps": torch.empty(1, dtype=torch.float64).pin_memory(),
                "post": torch.empty(6, dtype=torch.float64).pin_memory(),
                "counts": torch.empty(len(pv.lambdas), dtype=torch.uint64).pin_memory(),
                "p": torch.empty(len(pv.lambdas), dtype=torch.float64).pin_memory()}
    h2d = lam_host.numel() * 8
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())

    def e2e_step():
        lam_dev.copy_(lam_host, non_blocking=True)
        step()
        for key in ("idx", "rec", "n_acc", "eps", "post"):
            host_out[key].copy_(sel_out[key], non_blocking=True)
        for key in ("counts", "p"):
            host_out[key].copy_(pv_out[key], non_blocking=True)
        stream.synchronize()

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = units / e2e_s

    # Roofline of the dominant kernel (em_ou_fused_x2): 2 MUFU-class operations
    # (log, sqrt, sin, cos per Box-Muller pair) per path-step against 16 MUFU
    # lanes per SM per clock on the device's SMs at its maximum SM clock.
    em_avg_s = statistics.mean(em_ms) / 1e3
    achieved = abc_steps / em_avg_s / 1e9
    peak = (dev_props["sm_count"] * MUFU_PER_SM_CLK * dev_props["sm_max_mhz"] * 1e6
            / MUFU_PER_PATH_STEP / 1e9)
    roof = {"kernel": "em_ou_fused_x2", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "Gpath-steps/s", "frac": achieved / peak, "traffic": profiled_traffic(N),
            "peak_basis": (f"FP32+MUFU roofline: 2 MUFU ops/path-step (log,sqrt,sin,cos per pair), "
                           f"16 MUFU/SM/clk x {dev_props['sm_count']} SMs x {dev_props['sm_max_mhz']:g} MHz "
                           "(read from the device); FP32 pipe bound (6 ops/step, 128/SM/clk) is looser"),
            "pipe_bounds": pipe_bounds(statistics.mean(em_ms), abc_steps, dev_props)}
    clock = clocks.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)", "config": config_dict(abc, pv, world, k_global),
            "parts": {"em_ms_per_step": statistics.mean(em_ms),
                      "abc_path_steps": abc_steps, "pvalue_path_steps": pv_steps},
            "roofline": roof, "clocks": clock, "device": dev_props,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps}
    if world > 1:
        line["merge"] = {"k_global": k_global, "k_local": k_local,
                         "global_eps": float(merged["eps"].item()),
                         "global_n_acc": int(merged["n_acc"].item()),
                         "global_posterior_mean": [float(v) for v in merged["post"][:3].tolist()],
                         "note": "global accepted set of the N x world-sample job, merged over NCCL"}
    if world == 1 and not args.no_latency:
        # The latency half of the metric (BASELINE config 4, shortened replay)
        # and the batched-vs-plain form (config 3), each with its clocks.
        with ClockSampler(local_rank) as c_batch:
            batch = batch_comparison(args.jobs, args.batch_repeats)
        batch["clocks"] = c_batch.summary()
        with ClockSampler(local_rank) as c_serve:
            serve = serve_comparison(args.serve_rate, args.latency_serve_seconds, args.slots)
        serve["clocks"] = c_serve.summary()
        line["batch"] = batch
        line["serve"] = serve
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(abc, pv, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def job_specs(jobs):
    return [{"model": j.model, "y_obs": j.y_obs, "n_samples": j.n, "seed": j.seed, "k": j.k_accept}
            for j in jobs]


def batch_comparison(n_jobs, reps, clocks=None):
    """The uneven job mix run plain (one job per launch pair, one stream) and
    batched (one persistent, graph-replayed launch): `reps` alternating
    repeats of each, CUDA-event timed; the two forms give the same accepted
    sets, checked on the last repeat."""
    import torch
    from paper_1902_09046_gb300 import autotune, binding

    jobs = workloads.batched_jobs(n_jobs)
    specs = job_specs(jobs)
    total_steps = sum(j.path_steps for j in jobs)
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    max_n = max(j.n for j in jobs)
    dist = torch.empty(max_n, dtype=torch.float64, device=dev)
    ws = torch.empty(binding.abc_select_workspace_bytes(max_n), dtype=torch.uint8, device=dev)
    outs = [{"idx": torch.empty(j.k_accept, dtype=torch.uint32, device=dev),
             "rec": torch.empty((j.k_accept, 4), dtype=torch.float32, device=dev),
             "n_acc": torch.empty(1, dtype=torch.uint64, device=dev),
             "eps": torch.empty(1, dtype=torch.float64, device=dev),
             "post": torch.empty(6, dtype=torch.float64, device=dev)} for j in jobs]

    def plain():
        for j, o in zip(jobs, outs):
            binding.abc_prior_predictive(j.model, j.y_obs, j.n, j.seed, want_theta=False,
                                         out={"dist": dist[:j.n]}, stream=stream)
            binding.abc_select(dist[:j.n], k=j.k_accept, model=j.model, seed=j.seed,
                               workspace=ws, out=o, stream=stream)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b)

    with torch.cuda.stream(stream):
        t_tune = time.perf_counter()
        tile = autotune.tune(specs)
        t_tune = time.perf_counter() - t_tune
        batch = binding.Batch(specs, tile=tile, stream=stream)
        plain()
        batch.launch(graph=True, stream=stream)
        stream.synchronize()
        ms_plain, ms_batch = [], []
        for _ in range(reps):
            ms_plain.append(timed(plain))
            ms_batch.append(timed(lambda: batch.launch(graph=True, stream=stream)))
        same = True
        for o, r in zip(outs, batch.results()):
            same &= bool(torch.equal(o["idx"], r["idx"])) and bool(torch.equal(o["post"], r["post"]))
        batch.close()
    ratios = [p / b for p, b in zip(ms_plain, ms_batch)]
    plain_ms, batch_ms = statistics.median(ms_plain), statistics.median(ms_batch)
    return {"value": total_steps / (batch_ms / 1e3), "plain_value": total_steps / (plain_ms / 1e3),
            "unit": UNIT, "speedup_median": statistics.median(ratios), "speedup_min": min(ratios),
            "speedup_max": max(ratios), "batch_ms": batch_ms, "plain_ms": plain_ms,
            "batch_ms_range": [min(ms_batch), max(ms_batch)], "plain_ms_range": [min(ms_plain), max(ms_plain)],
            "repeats": reps, "path_steps": total_steps, "jobs": len(jobs), "tile": list(tile),
            "autotune_s": t_tune, "results_identical": same,
            "workload": (f"{len(jobs)} OU-ABC jobs, N log-uniform [1e3,1e7], S uniform {{100..10^4}}, "
                         "dt=10/S, 1% accepted; plain = one job per launch pair on one stream")}


def batch_mode(args):
    """256 uneven OU-ABC jobs: one job per launch pair (plain) against one
    persistent, graph-replayed launch (batched); same results either way."""
    import torch
    from paper_1902_09046_gb300 import binding
    from paper_1902_09046_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    binding.device_check()
    with ClockSampler(0) as clocks:
        res = batch_comparison(args.jobs, args.steps)
    line = {"mode": "batch", "metric": "EM path-steps/sec, batched vs plain", **res,
            "steps": args.steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": res.pop("workload")}, "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


def serve_comparison(rate, seconds, slots):
    """Poisson arrivals of mixed ABC / p-value jobs replayed in real time
    against the server with `slots` streams (served) and with one stream
    (plain, one job at a time); p50/p99 latency and aggregate throughput of
    each, and whether every job's result is the same in both."""
    import threading as th

    from paper_1902_09046_gb300 import binding

    jobs = workloads.served_jobs(rate_per_s=rate, duration_s=seconds)
    reqs = [binding.abc_request(j.model, j.y_obs, j.n, j.k_accept, j.seed) if j.kind == "abc"
            else binding.pvalue_request(j.lam, j.n_obs, j.n, j.ybar_obs, j.seed) for j in jobs]
    total_steps = sum(j.path_steps for j in jobs)
    arena = 64 << 30

    def run(n_slots):
        with binding.Server(arena, n_slots=n_slots) as srv:
            # warm-up: a few jobs of each kind
            for r in reqs[:8]:
                srv.release(srv.wait(srv.submit(r), 120.0)["job_id"])
            ids = [None] * len(jobs)
            t0 = time.perf_counter()

            def client():
                for i, (j, r) in enumerate(zip(jobs, reqs)):
                    delay = j.arrival_s - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                    ids[i] = srv.submit(r)

            c = th.Thread(target=client)
            c.start()
            c.join()
            res = [srv.wait(i, 600.0) for i in ids]
            t_end = time.perf_counter()
            lat = np.array([r["t_done"] - r["t_submit"] for r in res])
            first = min(r["t_submit"] for r in res)
            last = max(r["t_done"] for r in res)
            st = srv.stats()
            for i in ids:
                srv.release(i)
        ok = all(r["status"] == binding.PPABC_OK for r in res)
        kinds = np.array([j.kind == "abc" for j in jobs])
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "p99_abc_ms": float(np.percentile(lat[kinds], 99) * 1e3),
                "p99_pvalue_ms": float(np.percentile(lat[~kinds], 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
                "throughput": total_steps / (last - first), "makespan_s": last - first,
                "wall_s": t_end - t0, "all_ok": ok, "peak_arena_bytes": st["peak_arena_bytes"],
                "results": [(r["n_acc"], r["eps"], r["count"]) for r in res]}

    served = run(slots)
    plain = run(1)
    same = served.pop("results") == plain.pop("results")
    return {"served": served, "plain": plain, "slots": slots, "jobs": len(jobs), "path_steps": total_steps,
            "results_identical": same, "offered_path_steps_per_s": total_steps / seconds,
            "unit": "ms (latency), path-steps/s (throughput)",
            "workload": (f"Poisson {rate:g}/s for {seconds:g} s, 70% OU-ABC (N log-U[1e3,1e6], S U{{100..2000}}), "
                         "30% p-value (n=50, M log-U[1e4,1e6], lambda log-U[0.01,100]), HBM arena 64 GiB")}


def serve_mode(args):
    import torch
    from paper_1902_09046_gb300 import binding
    from paper_1902_09046_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    binding.device_check()
    with ClockSampler(0) as clocks:
        res = serve_comparison(args.serve_rate, args.serve_seconds, args.slots)
    line = {"mode": "serve", "metric": "p50/p99 job latency and aggregate path-steps/s, served vs plain",
            "value": res["served"]["p99_ms"], "higher_is_better": False, **res,
            "config": {"workload": res.pop("workload")}, "data": "synthetic (seeded)", "dtype": "f32",
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


PAPER_TOGGLE_SECONDS = 69.0  # N=8064, T=600, C=8000 on a Xeon Gold 6140 (AVX-512, P=16)


def toggle_mode(args):
    """The paper's benchmark: N = 8064 toggle-switch prior-predictive samples,
    T = 600 time points, C = 8000 cells, with the 19-quantile summaries and the
    distance to an observed target; cell-steps per second."""
    import torch
    from paper_1902_09046_gb300 import binding
    from paper_1902_09046_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    binding.device_check()
    dev_props = device_props(binding)
    N, model = 8064, workloads.toggle_model()
    q = workloads.toggle_observed_quantiles()
    cell_steps = N * model["C"] * (model["T"] - 1)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        binding.toggle_prior_predictive(model, q, N, 1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(0) as clocks:
        for a, b in ev:
            a.record(stream)
            binding.toggle_prior_predictive(model, q, N, 1)
            b.record(stream)
        torch.cuda.synchronize()
    ms = statistics.median([a.elapsed_time(b) for a, b in ev])
    # Roofline: per cell-step the method needs 2 normals (1 Box-Muller pair: log, sqrt, sin,
    # cos = 4 MUFU-class operations) and 2 powers (log2 + exp2 each) and 2 divisions
    # (reciprocal each): 10 MUFU-class operations at 16 per SM per clock.
    peak = dev_props["sm_count"] * MUFU_PER_SM_CLK * dev_props["sm_max_mhz"] * 1e6 / 10.0 / 1e9
    achieved = cell_steps / (ms / 1e3) / 1e9
    line = {"mode": "toggle", "metric": "toggle-switch prior-predictive cell-steps/s",
            "roofline": {"kernel": "toggle_abc", "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "Gcell-steps/s", "frac": achieved / peak,
                         "peak_basis": ("10 MUFU-class ops per cell-step (Box-Muller pair 4, two "
                                        f"powers 4, two divisions 2) at 16/SM/clk x {dev_props['sm_count']} SMs x "
                                        f"{dev_props['sm_max_mhz']:g} MHz")},
            "unit": "cell-steps/s", "value": cell_steps / (ms / 1e3), "ms_per_run": ms,
            "higher_is_better": True, "vs_baseline": (PAPER_TOGGLE_SECONDS * 1e3) / ms,
            "baseline": "paper Table A.1: 69 s for this workload, C with AVX-512, 16 cores",
            "dtype": "f32", "data": "synthetic (seeded)", "steps": args.steps,
            "config": {"workload": "toggle switch N=8064 T=600 C=8000, 19 quantiles + distance"},
            "clocks": clocks.summary(), "device": dev_props}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        thr = oracle.default_threads()
        n_cpu = 2 * thr
        t0 = time.perf_counter()
        oracle.toggle_prior_predictive(model, q, n_cpu, 1, want_theta=False, want_summ=False,
                                       n_threads=thr)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n_cpu * model["C"] * (model["T"] - 1) / dt,
                                "unit": "cell-steps/s", "cores": thr, "kind": "oracle",
                                "sample": f"{n_cpu} of the 8064 samples, FP64, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0




def bege_profile(launch_ms, particle_steps, dev):
    """Per-pipe ceilings of bege_density from its measured cycles per
    particle-step on one SM sub-partition (issue slots, FMA pipe and its heavy
    half, ALU pipe), read from the committed ncu summary, with the achieved
    rate's fraction of each; None if absent or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "bege_density_counts.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for rel in BEGE_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    cyc = rec.get("cycles_per_particle_step")
    if rec.get("source_hash") != h.hexdigest()[:16] or not cyc:
        return None
    achieved = particle_steps / (launch_ms / 1e3)
    smsp_cycles_per_s = dev["sm_count"] * 4 * dev["sm_max_mhz"] * 1e6
    out = {"cycles_per_particle_step": cyc}
    for name, c in cyc.items():
        if name == "elapsed":
            continue
        ceiling = smsp_cycles_per_s / c
        out[name] = {"ceiling_particle_steps_per_s": ceiling, "frac": achieved / ceiling}
    out["binding"] = min((k for k in out if k != "cycles_per_particle_step"),
                         key=lambda k: out[k]["ceiling_particle_steps_per_s"])
    return out


BEGE_SOURCES = ("paper_1902_09046_gb300/csrc/bege.cu", "paper_1902_09046_gb300/csrc/dfloat.cuh")


def bege_mode(args):
    """BEGE log-likelihoods (Sec. 4.2) of 1024 particles on a 1099-month
    return series, as in one SMC iteration of the paper's BEGE inference:
    particle-months per second, for particles drawn from the prior (the first
    iteration) and particles concentrated around a plausible parameter vector
    (a later iteration)."""
    import torch
    from paper_1902_09046_gb300 import binding
    from paper_1902_09046_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    binding.device_check()
    dev_props = device_props(binding)
    r_np = workloads.bege_returns()
    T, n_p, h = len(r_np), workloads.BEGE_N_PARTICLES, workloads.BEGE_H
    sets = {"later": workloads.bege_particles(n_p, seed=6, centre=workloads.BEGE_THETA_REF, rel_spread=0.05),
            "prior": workloads.bege_particles(n_p, seed=6)}
    r = torch.from_numpy(r_np).cuda()
    stream = torch.cuda.current_stream()
    res = {}
    with ClockSampler(0) as clocks:
        for name, th_np in sets.items():
            th = torch.from_numpy(th_np).cuda()
            out = binding.bege_loglik(th, r, h)
            for _ in range(max(3, args.warmup)):
                binding.bege_loglik(th, r, h, out=out)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for a, b in ev:
                a.record(stream)
                binding.bege_loglik(th, r, h, out=out)
                b.record(stream)
            torch.cuda.synchronize()
            ms = statistics.median([a.elapsed_time(b) for a, b in ev])
            ll = out["ll"].cpu().numpy()
            res[name] = {"ms": ms, "particle_steps_per_s": n_p * T / (ms / 1e3),
                         "finite": int(np.isfinite(ll).sum())}
    main = res["later"]
    prof = bege_profile(main["ms"], n_p * T, dev_props)
    if prof:
        bind = prof[prof["binding"]]
        roof = {"kernel": "bege_density", "bound": "alu", "unit": "particle-steps/s",
                "achieved": main["particle_steps_per_s"], "peak": bind["ceiling_particle_steps_per_s"],
                "frac": bind["frac"], "traffic": None, "pipe_bounds": prof,
                "peak_basis": (f"{prof['binding']} ceiling: {dev_props['sm_count']} SMs x 4 sub-partitions x "
                               f"{dev_props['sm_max_mhz']:g} MHz / measured cycles per particle-step "
                               "(profiles/bege_density_counts.json)")}
    else:
        roof = {"kernel": "bege_density", "bound": "alu", "unit": "particle-steps/s",
                "achieved": main["particle_steps_per_s"], "peak": None, "frac": None, "traffic": None,
                "peak_basis": "no current ncu summary for this kernel"}
    line = {"mode": "bege", "metric": "BEGE log-likelihood particle-months/s", "unit": "particle-steps/s",
            "value": main["particle_steps_per_s"], "ms_per_run": main["ms"], "higher_is_better": True,
            "vs_baseline": None, "dtype": "f64 sums, double-float (2 x f32) per node", "data": "synthetic (seeded)",
            "steps": args.steps, "runs": res, "roofline": roof,
            "config": {"workload": f"BEGE log-likelihood, {n_p} particles x T={T} months, N_w=100, h={h:g}; "
                                   "'later' = particles within 5% of the prior box around a plausible "
                                   "vector, 'prior' = prior draws"},
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        thr = oracle.default_threads()
        n_cpu = 4 * thr
        t0 = time.perf_counter()
        oracle.bege_loglik(sets["later"][:, :n_cpu], r_np, h, n_threads=thr)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n_cpu * T / dt, "unit": "particle-steps/s", "cores": thr,
                                "kind": "oracle", "sample": f"{n_cpu} of the 1024 'later' particles, FP64, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def configs_mode(args):
    """Each synthetic configuration timed on its own (GPU, CUDA events, median
    of --steps after warm-up), with the oracle on a bounded sample of it."""
    import torch
    import oracle
    from paper_1902_09046_gb300 import binding
    from paper_1902_09046_gb300 import build as libbuild

    torch.cuda.set_device(0)
    libbuild.build()
    oracle.build()
    binding.device_check()
    thr = oracle.default_threads()
    stream = torch.cuda.current_stream()

    def gpu_ms(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.median([a.elapsed_time(b) for a, b in ev])

    rows = []
    for name, w in (("ou_abc_n1e4_s1e3", workloads.abc_small()), ("ou_abc_n2p24_s1e4", workloads.abc_large())):
        ws = torch.empty(binding.abc_select_workspace_bytes(w.n_samples), dtype=torch.uint8, device="cuda")
        dist = torch.empty(w.n_samples, dtype=torch.float64, device="cuda")

        def run(w=w, ws=ws, dist=dist):
            binding.abc_prior_predictive(w.model, w.y_obs, w.n_samples, w.seed, want_theta=False,
                                         out={"dist": dist})
            binding.abc_select(dist, k=w.k_accept, model=w.model, seed=w.seed, workspace=ws)
        ms = gpu_ms(run)
        steps = w.n_samples * w.model["n_steps"]
        n_cpu = min(w.n_samples, max(thr * 16, int(2e8 / w.model["n_steps"])))
        t0 = time.perf_counter()
        oracle.ou_prior_predictive(w.model, w.y_obs, n_cpu, w.seed, want_theta=False, n_threads=thr)
        cpu_s = time.perf_counter() - t0
        rows.append({"config": name, "gpu_ms": ms, "gpu_path_steps_per_s": steps / (ms / 1e3),
                     "oracle_path_steps_per_s": n_cpu * w.model["n_steps"] / cpu_s,
                     "oracle_sample": f"{n_cpu} samples", "oracle_cores": thr})
    pv = workloads.pvalue_sweep_workload()
    lam = torch.from_numpy(pv.lambdas).cuda()
    ms = gpu_ms(lambda: binding.pvalue_sweep(lam, pv.n_obs, pv.m_sets, pv.ybar_obs, pv.seed))
    steps = len(pv.lambdas) * pv.m_sets * (pv.n_obs + 1)
    m_cpu = 20_000
    t0 = time.perf_counter()
    oracle.pvalue_sweep(pv.lambdas, pv.n_obs, m_cpu, pv.ybar_obs, pv.seed, n_threads=thr)
    cpu_s = time.perf_counter() - t0
    rows.append({"config": "pvalue_k64_n50_m1e6", "gpu_ms": ms, "gpu_path_steps_per_s": steps / (ms / 1e3),
                 "oracle_path_steps_per_s": len(pv.lambdas) * m_cpu * (pv.n_obs + 1) / cpu_s,
                 "oracle_sample": f"M={m_cpu} per lambda", "oracle_cores": thr})
    # Algorithm 2 (weak-informativity cut-offs): 64 lambdas x 2 x 16384 data sets of n = 50
    wl = torch.from_numpy(workloads.pvalue_lambdas()).cuda()
    N2 = binding.WEAKINF_MAX_SETS
    ms = gpu_ms(lambda: binding.weakinf_test(wl, 1.0, 50, N2, 0.05, 9))
    steps = 64 * 2 * N2 * 51
    t0 = time.perf_counter()
    oracle.weakinf(workloads.pvalue_lambdas()[:8], 1.0, 50, 2048, 0.05, 9, n_threads=thr)
    cpu_s = time.perf_counter() - t0
    rows.append({"config": "weakinf_k64_n50_N16384", "gpu_ms": ms, "gpu_path_steps_per_s": steps / (ms / 1e3),
                 "oracle_path_steps_per_s": 8 * 2 * 2048 * 51 / cpu_s,
                 "oracle_sample": "8 lambdas, N=2048 (its N^2 comparisons included)", "oracle_cores": thr})
    # Algorithm 1 as stated: the first 10^4 acceptances at ~1% acceptance (OU, 1000 steps)
    w = workloads.abc_small()
    _, _, d_o = oracle.ou_prior_predictive(w.model, w.y_obs, 20_000, w.seed, n_threads=thr)
    eps = float(np.quantile(d_o, 0.01))
    res = {}

    def rej():
        res.update(binding.abc_rejection(w.model, w.y_obs, eps, 10_000, 1 << 22, w.seed, chunk=1 << 18))
    ms = gpu_ms(rej)
    rows.append({"config": "abc_rejection_ou_s1e3_m1e4", "gpu_ms": ms,
                 "gpu_path_steps_per_s": res["tried"] * w.model["n_steps"] / (ms / 1e3),
                 "proposals": res["tried"], "accepted": res["n_acc"],
                 "note": "wall time includes the host check of the count every 4 chunks"})
    # ABC recalibration of the small ABC's accepted sample: its 10^4 stored
    # pairs, the 100 accepted, 100 neighbours each
    out = binding.abc_prior_predictive(w.model, w.y_obs, w.n_samples, w.seed, want_theta=True, want_summ=True)
    sel = binding.abc_select(out["dist"], k=w.k_accept, theta=out["theta"])
    torch.cuda.synchronize()
    ms = gpu_ms(lambda: binding.abc_recalibrate(out["summ"], out["theta"], sel["idx"], 100))
    summ_h, th_h, acc_h = (out["summ"].cpu().numpy(), out["theta"].cpu().numpy(),
                           sel["idx"].cpu().numpy().astype(np.uint32))
    t0 = time.perf_counter()
    oracle.recalibrate(summ_h, th_h, acc_h, 100, n_threads=thr)
    cpu_s = time.perf_counter() - t0
    rows.append({"config": "abc_recalibrate_n1e4_q100_k100", "gpu_ms": ms, "oracle_ms": 1e3 * cpu_s,
                 "oracle_cores": thr, "note": "not a path-step workload: n x q distances and q selections"})
    print(json.dumps({"mode": "configs", "unit": UNIT, "rows": rows}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.mode == "batch":
        return batch_mode(args)
    if args.mode == "serve":
        return serve_mode(args)
    if args.mode == "toggle":
        return toggle_mode(args)
    if args.mode == "bege":
        return bege_mode(args)
    if args.mode == "configs":
        return configs_mode(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
