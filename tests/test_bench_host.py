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


def test_sub_workloads_keep_the_family_and_parameters():
    """The CPU samples run the benchmark workload's own family and parameters on a smaller box."""
    big = bench.workload("droplet512")
    small = bench.sub_workload("droplet512", 40 ** 3)
    assert (small.nx, small.ny, small.nz) == (40, 40, 40) and small.radius == 10.0
    for k in ("rho_l", "rho_g", "mu_l", "mu_g", "sigma", "width", "mobility", "wall_z"):
        assert getattr(small, k) == getattr(big, k), k
    b = bench.sub_workload("rising_bubble", 2 * 32 ** 3)
    ref = bench.workload("rising_bubble")
    assert (b.nx, b.ny, b.nz) == (32, 32, 64) and b.wall_z == 1
    # the bubble keeps its dimensionless groups (ratios, Eo, Mo), so sigma, g and mu follow R
    for k in ("rho_l", "rho_g", "width", "mobility"):
        assert getattr(b, k) == getattr(ref, k), k
    assert b.mu_l / b.mu_g == pytest.approx(ref.mu_l / ref.mu_g)


def test_large_boxes_take_the_traffic_of_their_proxy_scaled_per_node(monkeypatch, tmp_path):
    """The 512^3 droplet (too large for a multi-pass ncu capture) reads the 256^3 droplet's summary
    of the same kernel, scaled per node; a summary of its own would take precedence."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "ab" * 32)
    (prof / "lbm_kernel_static_droplet_256.txt").write_text(
        "kernel: lbm_kernel\nnodes: 1000\nsource_sha256: " + "ab" * 32 + "\ndram_bytes_per_launch: 240000\n")
    assert bench.measured_traffic("lbm_kernel", "droplet512", 8000) == pytest.approx(1920000)
    assert bench.traffic_source("lbm_kernel", "droplet512")[1] == "droplet256"
    (prof / "lbm_kernel_static_droplet_512.txt").write_text(
        "nodes: 8000\nsource_sha256: " + "ab" * 32 + "\ndram_bytes_per_launch: 2000000\n")
    assert bench.measured_traffic("lbm_kernel", "droplet512", 8000) == pytest.approx(2000000)


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
    assert d["config"]["workload"] == "static_droplet_512^3"
    assert "sub-box of the workload" in d["config"]["sample"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    r = _reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
