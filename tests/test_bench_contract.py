"""The benchmark's JSON contract, checked on the CPU through its reference arm
(the oracle timed on the host cores), and the helpers that read the
committed ncu summaries."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REQUIRED = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def _run(args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_prints_one_contract_line():
    d = _run(["--impl", "reference", "--steps", "2", "--warmup", "1", "--abc-samples", "4096",
              "--abc-steps", "200", "--pv-sets", "2000"])
    assert REQUIRED <= set(d), REQUIRED - set(d)
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "path-steps/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("ou_abc N=4096 S=200")


def test_committed_profiles_match_the_kernel_sources():
    """bench.py reads DRAM traffic, per-pipe cycles and FP64 counts from the
    committed ncu summaries only while their source hashes match; a kernel
    change must come with a new capture."""
    sys.path.insert(0, ROOT)
    import bench
    traffic = json.load(open(os.path.join(ROOT, "profiles", "em_ou_fused_traffic.json")))
    assert traffic["source_hash"] == bench.kernel_source_hash()
    gb300 = {"sm_count": 152, "sm_max_mhz": 2070.0}
    pb = bench.pipe_bounds(200.0, 16777216 * 10000, gb300)
    assert pb is not None and pb["binding"] in ("issue", "alu", "fma", "fmaheavy")
    if traffic["dram_bytes"] is None:  # the kernel changed since the last full-size DRAM capture
        assert bench.profiled_traffic(16777216) is None
    else:
        assert bench.profiled_traffic(16777216) == pytest.approx(traffic["dram_bytes"])
    assert bench.bege_profile(60.0, 1024 * 1099, gb300) is not None
