"""Host-side logic of bench.py that needs no GPU: the ncu traffic lookup and its source-hash
guard, and the reference arm (the FP64 oracle) with its JSON line."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_BUBBLE = 128 * 128 * 256


def test_committed_profile_traffic_is_within_the_algorithmic_bytes():
    """A step kernel's committed ncu summary, when it was taken on the current sources, gives DRAM
    traffic per node between the kernel's L2-served floor and its algorithmic bytes (more would
    mean wasted re-reads).  Summaries of changed kernels are ignored, as bench.py ignores them."""
    checked = 0
    for kernel, store, lo, hi in (("lbm_kernel", "fp32", 200, 256), ("lbm16_kernel", "bf16", 120, 156),
                                  ("lbm_mom_kernel", "mom", 90, 120), ("lbm_mom_kernel", "mom_bf16", 60, 88)):
        t = bench.measured_traffic(kernel, "rising_bubble", N_BUBBLE, store)
        if t is None:
            continue
        checked += 1
        assert lo <= t / N_BUBBLE <= hi, (kernel, store, t / N_BUBBLE)
    if checked == 0:
        pytest.skip("no committed ncu summary matches the current kernel sources")


def test_traffic_scales_with_nodes_and_is_dropped_when_sources_change(monkeypatch):
    t = bench.measured_traffic("lbm_kernel", "rising_bubble", N_BUBBLE)
    if t is not None:
        assert bench.measured_traffic("lbm_kernel", "rising_bubble", 2 * N_BUBBLE) == pytest.approx(2 * t)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "0" * 64)
    assert bench.measured_traffic("lbm_kernel", "rising_bubble", N_BUBBLE) is None
    assert bench.measured_traffic("lbm_kernel", "no_such_workload", N_BUBBLE) is None
    assert bench.measured_traffic("no_such_kernel", "rising_bubble", N_BUBBLE) is None


def _reference(env_extra, *extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                           "--warmup", "3", "--reference-seconds", "3", *extra],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)


def test_reference_arm_prints_one_oracle_line():
    r = _reference({})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["dtype"] == "f64"
    assert d["config"]["workload"] == "rising_bubble_128x128x256"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    r = _reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
