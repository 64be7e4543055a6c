#!/usr/bin/env python
"""Benchmark of the coupled TSLB + Allen-Cahn step on B300 (one JSON line on rank 0).

Workload (default): the static droplet in a periodic 512^3 box (134M nodes), R = 128 centred,
W = 4, density ratio 10, viscosity ratio 10, sigma = 0.01, fluid at rest, balanced initial
pressure; synthetic seeded inputs.  It is the largest single-GPU configuration of the MLUPS sweep
and the box of the paper's own performance tables (a 512^3 water-air box).  A step is one time
step of the whole box: two kernel launches by default (the z-marching Allen-Cahn kernel, then the
lattice Boltzmann kernel).  The state (16.6 GB of FP32 populations and fields per copy) is far
larger than the 126 MB L2, so consecutive steps stream from HBM and no flush is needed.

  value  MLUPS = nodes * K / device time of K steps (CUDA events on the solver's stream),
         summed over ranks (each rank runs its own replica: weak scaling).
  e2e    the same metric through the public API from pinned host buffers: init from host,
         K steps, observables and a read-back of phi, u, p to host, all inside the timed region.
  roofline  dominant kernel (the lattice Boltzmann kernel): algorithmic bytes per node update
         (FP32 256 B: read 27 g + phi + 3 u, write 27 g + 3 u + the 3-component Allen-Cahn flux;
         16-bit 156 B) over its mean launch duration, against the measured HBM copy peak; step_*
         the same for the whole step against the method's state (248 B / 148 B per node update:
         the state read once and written once; the flux this design carries is not counted).
  store_compare  the same workload with the other stores (BF16 / FP16 populations, FP32 / BF16 /
         FP16 moments), device-timed over min(K, 2000) steps.
  rising_bubble  the 128 x 128 x 256 rising bubble (walls on z, density ratio 1000, viscosity
         ratio 100, Eo = 10, Mo = 1e-4) with FP32 populations and with BF16 moments.
  ensemble  the batched ensemble of 256 seeded droplets (32^3 .. 96^3 boxes): autotuned, min(K, 400)
         steps from CUDA graphs, next to the same boxes advanced one context at a time.
  closure_network  the learned closure's network on the 64^3 coarse grid: device time of a forward
         pass (and its useful BF16 TFLOP/s against the measured tensor peak) and of a training step.
  cpu_baseline  the FP64 oracle (plain C, OpenMP) on the host cores, on a bounded sub-box of the
         same workload.

--impl reference runs the FP64 CPU oracle as the reference arm (rank 0 only).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes per node update of a whole step: the method's state read once and written once
#   FP32:   27 g + phi + 3 ubar floats = 124 B, twice
#   16-bit: 27 h (2 B) + P + phi + 3 ubar floats = 74 B, twice
# (the Allen-Cahn flux W that this design carries from the lattice Boltzmann kernel of one step
# to the Allen-Cahn kernel of the next, 24 B per node, is extra traffic and not counted here)
STEP_BYTES = {"fp32": 248, "bf16": 148, "fp16": 148, "mom": 112, "mom_bf16": 80, "mom_fp16": 80}
# algorithmic bytes per node of each kernel that can dominate a step
KERNEL_BYTES = {"lbm_kernel": 256,      # read 27 g + phi^{n+1} + 3 ubar, write 27 g + 3 ubar + 3 W
                "fused2_kernel": 248,
                "lbm16_kernel": 156,    # read 27 h + P + phi^{n+1} + 3 ubar, write 27 h + P + 3 ubar + 3 W
                "lbm_mom_kernel": 120,  # read 13 moments + phi^{n+1}, write 13 moments + 3 W
                "lbm_mom_plain_kernel": 120,
                "ac_div_kernel": 20}    # read phi^n + 3 W^n, write phi^{n+1}
STORES = {"fp32": 0, "bf16": 1, "fp16": 2, "mom": 3, "mom_bf16": 4, "mom_fp16": 5}
# floats (or their 16-bit share) of one copy of the state per node: g + phi + u, or h/2 + P + phi + u
STATE_FLOATS = {"fp32": 31, "bf16": 18.5, "fp16": 18.5, "mom": 14, "mom_bf16": 10, "mom_fp16": 10}
FALLBACK_HBM_GBS = 6400.0
METRIC = "MLUPS & % HBM peak: coupled LBM+Allen-Cahn step, FP32 vs BF16 store"
# sources that define each step kernel's device code (the profile of a kernel is reused only while
# these files are unchanged)
KERNEL_SOURCES = {
    "lbm_kernel": ["paper_2501_00846_b300/csrc/step_unfused.cu", "paper_2501_00846_b300/csrc/lbm_node.cuh",
                   "paper_2501_00846_b300/csrc/tslb_device.cuh"],
    "fused2_kernel": ["paper_2501_00846_b300/csrc/step_fused2.cu", "paper_2501_00846_b300/csrc/tslb_device.cuh"],
    "lbm16_kernel": ["paper_2501_00846_b300/csrc/step_lbm16.cu", "paper_2501_00846_b300/csrc/tslb_device.cuh"],
    "ac_div_kernel": ["paper_2501_00846_b300/csrc/step_split.cu", "paper_2501_00846_b300/csrc/ac_div.cuh",
                      "paper_2501_00846_b300/csrc/tslb_device.cuh"],
    "lbm_mom_kernel": ["paper_2501_00846_b300/csrc/step_mom.cu", "paper_2501_00846_b300/csrc/mom_tile.cuh",
                       "paper_2501_00846_b300/csrc/mom_device.cuh", "paper_2501_00846_b300/csrc/tslb_device.cuh"],
}
KERNEL_NAMES = {0: "lbm_kernel", 1: "lbm_kernel", 2: "fused2_kernel"}


# algorithmic bytes per node and launch of the moment kernel with 16-bit a and B: read p* + 5 packed
# words + 3 u + phi^{n+1}, write p* + 5 words + 3 u + 3 W
MOM16_KERNEL_BYTES = 88


def kernel_name(path, store):
    if store.startswith("mom"):
        return "lbm_mom_kernel" if path == 0 else "lbm_mom_plain_kernel"
    if store != "fp32":
        return "lbm16_kernel" if path == 0 else "lbm_kernel"
    return KERNEL_NAMES[path]
LAUNCHES_PER_STEP = {0: 2, 1: 3, 2: 1}


def workload(name):
    from paper_2501_00846_b300 import inputs
    if name == "rising_bubble":
        return inputs.rising_bubble()
    if name.startswith("droplet"):
        L = int(name[len("droplet"):])
        return inputs.static_droplet(L=L)
    raise SystemExit(f"unknown workload {name}")


def sub_workload(name, nodes):
    """A box of about `nodes` nodes of the same family and parameters as workload `name` (a
    droplet: L^3 with R = L/4; the bubble: L x L x 2L with R = L/4 at z = L/2), for the CPU
    oracle's bounded samples: the per-node arithmetic does not depend on the box size."""
    from paper_2501_00846_b300 import inputs
    if name.startswith("droplet"):
        L = int(max(8, min(int(name[len("droplet"):]), round(nodes ** (1 / 3)))))
        return inputs.static_droplet(L=L)
    L = int(max(8, min(128, round((nodes / 2) ** (1 / 3)))))
    return inputs.rising_bubble(nx=L, ny=L, nz=2 * L, R=max(1.5, L / 4), zc=L / 2)


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


# workloads too large for a multi-pass ncu capture take the DRAM traffic of the same kernel on a
# smaller box of the same family, scaled per node (per-node traffic does not depend on the box
# size once the state is far larger than L2)
TRAFFIC_PROXY = {"droplet512": "droplet256"}
PROFILE_NAMES = {"droplet512": "static_droplet_512", "droplet256": "static_droplet_256",
                 "droplet128": "static_droplet_128", "rising_bubble": "rising_bubble"}


def traffic_source(kernel, wl_name, store="fp32"):
    """(path of the committed ncu summary that measured_traffic reads, workload it was taken on)."""
    tag = kernel if store in ("fp32", "mom") else f"{kernel}_{store}"
    if store in ("mom_bf16", "mom_fp16"):
        tag = f"{kernel}_{store[4:]}"
    for name in (wl_name, TRAFFIC_PROXY.get(wl_name)):
        if name is None:
            continue
        path = os.path.join(ROOT, "profiles", f"{tag}_{PROFILE_NAMES.get(name, name)}.txt")
        if os.path.exists(path):
            return path, name
    return None, None


def measured_traffic(kernel, wl_name, nodes, store="fp32"):
    """DRAM bytes per launch of a step kernel from the committed ncu summary
    profiles/<kernel>[_<store>]_<workload>.txt (or of the workload's smaller proxy, scaled per
    node), if its source hash matches the current kernel sources (else None)."""
    if kernel not in KERNEL_SOURCES:
        return None
    path, _ = traffic_source(kernel, wl_name, store)
    if path is None:
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != kernel_source_hash(kernel):
        return None
    try:
        b = float(kv["dram_bytes_per_launch"])
        n = float(kv["nodes"])
    except (KeyError, ValueError):
        return None
    return b * nodes / n


def bf16_peak():
    """Dense BF16 tensor peak in TFLOP/s: the measured burst figure (a network pass is timed on its
    own), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1800.0


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5 and os.path.getsize(self.out.name) == 0:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.out.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 6:
                    rows.append(parts)
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(seconds, wl_name="droplet512", max_steps=None):
    """Time the FP64 oracle on a sub-box of workload wl_name (same family and parameters, so the
    same per-node arithmetic) for about `seconds`; returns (MLUPS, description, threads)."""
    import oracle
    wl = sub_workload(wl_name, 16 * 16 * 32)
    P = oracle.Params(**wl.params())
    s = oracle.init(P, wl.phi0(), wl.u0(), wl.pstar_init())
    t0 = time.perf_counter()
    s = oracle.run(P, s, 2)
    per_node = (time.perf_counter() - t0) / (2 * P.n)
    # choose the sub-box so that one step takes ~seconds/8
    wl = sub_workload(wl_name, max(P.n, min(128 * 128 * 256, seconds / 8 / per_node)))
    P = oracle.Params(**wl.params())
    s = oracle.init(P, wl.phi0(), wl.u0(), wl.pstar_init())
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and (max_steps is None or steps < max_steps):
        s = oracle.step(P, s)
        steps += 1
    dt = time.perf_counter() - t0
    desc = (f"oracle on a {wl.nx}x{wl.ny}x{wl.nz} sub-box of the benchmark workload (same family and "
            f"parameters), {steps} steps in {dt:.1f} s")
    return P.n * steps / dt / 1e6, desc, oracle.get_threads()


def replica_max(x, world, device):
    """The largest of the ranks' values of x (the slowest replica bounds the job); x itself on one
    rank.  Collective over the default process group when world > 1."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(n_nodes, steps, seconds, world):
    """Whole-job MLUPS of `world` replicas that each advanced n_nodes nodes `steps` times, timed by
    the slowest (seconds = the max over ranks)."""
    return world * n_nodes * steps / seconds / 1e6


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, each step on a bounded sub-box of the workload."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    budget = args.reference_seconds
    # calibrate the per-node cost, then size the sub-box so warmup + steps fit the budget
    wl = sub_workload(args.workload, 16 * 16 * 32)
    P = oracle.Params(**wl.params())
    s = oracle.init(P, wl.phi0(), wl.u0(), wl.pstar_init())
    t0 = time.perf_counter()
    oracle.run(P, s, 2)
    per_node = (time.perf_counter() - t0) / (2 * P.n)
    wl = sub_workload(args.workload, budget / max(1, args.steps + args.warmup) / per_node)
    P = oracle.Params(**wl.params())
    s = oracle.init(P, wl.phi0(), wl.u0(), wl.pstar_init())
    s = oracle.run(P, s, args.warmup)
    t0 = time.perf_counter()
    s = oracle.run(P, s, args.steps)
    dt = time.perf_counter() - t0
    value = P.n * args.steps / dt / 1e6
    desc = (f"each step: one oracle step of a {wl.nx}x{wl.ny}x{wl.nz} sub-box of the workload "
            "(same family and parameters)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload(args.workload).name, "sample": desc},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args, stream):
    """The batched ensemble: 256 seeded static droplets in uneven periodic boxes (32^3 .. 96^3,
    density ratios 10 .. 1000), autotuned, K_e steps replayed from CUDA graphs, device-timed, with
    FP32 populations and with BF16 moments; beside it the same boxes advanced one context at a time
    (each box's two kernels launched separately), device-timed over fewer steps."""
    import numpy as np
    import torch
    from paper_2501_00846_b300 import inputs, solver
    wls = inputs.droplet_ensemble()
    n_nodes = sum(wl.n for wl in wls)
    ke = min(args.steps, 400)
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
    fields = [(f32(wl.phi0()), f32(wl.u0()), f32(wl.pstar_init())) for wl in wls]

    def batched(storage, persistent=False):
        """Autotuned batched run of every box with one storage: (ms per ke steps, tuning, boxes
        that went non-finite).  persistent: one cooperative launch per step instead of the two
        graph-replayed launches."""
        e = solver.Ensemble([dict(wl.params(), storage=storage) for wl in wls], stream=stream)
        for b, (phi0, u0, ps0) in enumerate(fields):
            e.init_fields(b, phi0, u0, ps0)
        e.step(2)
        tun = e.autotune(reps=3)
        e.set_persistent(persistent)
        e.step(16)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e.step(ke)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        bad = sum(e.observables(b, allow_nonfinite=True)["n_nonfinite"] > 0 for b in range(len(wls)))
        e.close()
        return ms, tun, bad

    with torch.cuda.stream(stream):
        ms, tun, bad = batched(solver.LBM_FP32)
        ms_m, tun_m, bad_m = batched(solver.LBM_MOM_BF16)
        ms_p, _, bad_p = batched(solver.LBM_FP32, persistent=True)
        ms_pm, _, bad_pm = batched(solver.LBM_MOM_BF16, persistent=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the same boxes one context each, every box stepped in turn
        ku = 20
        ctxs = []
        for wl, (phi0, u0, ps0) in zip(wls, fields):
            c = solver.Solver(stream=stream, **wl.params())
            c.init_fields(phi0, u0, ps0)
            ctxs.append(c)
        for c in ctxs:
            c.step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ku):
            for c in ctxs:
                c.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_u = e0.elapsed_time(e1)
        for c in ctxs:
            c.close()
    value = n_nodes * ke / (ms * 1e-3) / 1e6
    unbatched = n_nodes * ku / (ms_u * 1e-3) / 1e6
    return {"workload": "256 static droplets, periodic cubes L in [32, 96], R in [6, L/4], sigma in "
                        "[0.001, 0.02], density ratio log-uniform in [10, 1000], seed 2501",
            "nodes": n_nodes, "value": value, "unit": "MLUPS", "steps": ke, "ms_per_step": ms / ke,
            "launches_per_step": 2, "graph_steps": tun["graph_steps"],
            "tuning": {k: tun[k] for k in ("lbm_block", "ac_rows", "ac_zlen", "lbm_us", "ac_us")},
            "unbatched": {"value": unbatched, "unit": "MLUPS", "steps": ku, "ms_per_step": ms_u / ku,
                          "launches_per_step": 2 * len(wls)},
            "speedup": value / unbatched, "boxes_nonfinite": int(bad),
            "bf16_moments": {"value": n_nodes * ke / (ms_m * 1e-3) / 1e6, "unit": "MLUPS", "steps": ke,
                             "ms_per_step": ms_m / ke, "ac_us": tun_m["ac_us"], "lbm_us": tun_m["lbm_us"],
                             "boxes_nonfinite": int(bad_m)},
            "persistent": {"launches_per_step": 1,
                           "fp32": {"value": n_nodes * ke / (ms_p * 1e-3) / 1e6, "unit": "MLUPS", "steps": ke,
                                    "ms_per_step": ms_p / ke, "boxes_nonfinite": int(bad_p)},
                           "bf16_moments": {"value": n_nodes * ke / (ms_pm * 1e-3) / 1e6, "unit": "MLUPS",
                                            "steps": ke, "ms_per_step": ms_pm / ke, "boxes_nonfinite": int(bad_pm)}}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="droplet512")
    ap.add_argument("--path", type=int, default=0,
                    help="step launch: 0 two kernels (default), 1 three kernels, 2 one fused kernel")
    ap.add_argument("--split", type=int, default=0, help="work split of the fused kernel (0 = default)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="CPU time budget of the reference arm (warm-up and timed steps together)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--store", default="fp32", choices=list(STORES),
                    help="population storage of the headline line (the others go to store_compare)")
    ap.add_argument("--no-store-compare", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 256-droplet batched ensemble")
    ap.add_argument("--no-bubble", action="store_true", help="skip the rising bubble beside a droplet workload")
    ap.add_argument("--no-closure", action="store_true", help="skip timing the learned closure's network")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2501_00846_b300 import solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    wl = workload(args.workload)
    N = wl.n
    # an explicit stream: the library enqueues every kernel on it and the events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def fields_of(w):
        return (np.ascontiguousarray(w.phi0(), np.float32), np.ascontiguousarray(w.u0(), np.float32),
                np.ascontiguousarray(w.pstar0(), np.float32))

    phi0, u0, ps0 = fields_of(wl)

    def device_timed(store, steps, sampler=None, w=None, fields=None):
        """K steps of one store on the device, CUDA events on the solver's stream; then the
        dominant kernel alone (paths 0 and 1: the lattice Boltzmann kernel relaunched without
        advancing the state; path 2: the step is one kernel).  w, fields: another workload and
        its initial fields (default: the benchmark workload).  Returns (ms of K steps, ms per
        dominant-kernel launch, observables after the K steps, the solver)."""
        w = wl if w is None else w
        f_phi, f_u, f_ps = (phi0, u0, ps0) if fields is None else fields
        s = solver.Solver(stream=stream, storage=STORES[store], **w.params())
        s.set_path(args.path)
        s.set_split(args.split)
        s.init_fields(f_phi, f_u, f_ps)
        s.step(args.warmup)
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        kernel_ms = ms / steps
        if args.path in (0, 1):
            nrep = min(steps, 1000)
            s.run_phase(0, 1)
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            s.run_phase(1, nrep)
            k1.record(stream)
            torch.cuda.synchronize()
            kernel_ms = k0.elapsed_time(k1) / nrep
        obs = s.observables(allow_nonfinite=True)
        return ms, kernel_ms, obs, s

    def roofline(store, ms_step, kernel_ms, wl_name=None, nodes=None):
        wl_name = args.workload if wl_name is None else wl_name
        nodes = N if nodes is None else nodes
        kernel = kernel_name(args.path, store)
        kbytes = MOM16_KERNEL_BYTES if store in ("mom_bf16", "mom_fp16") else KERNEL_BYTES[kernel]
        achieved = kbytes * nodes / (kernel_ms * 1e-3) / 1e9
        step_gbs = STEP_BYTES[store] * nodes / (ms_step * 1e-3) / 1e9
        traffic = measured_traffic(kernel, wl_name, nodes, store)
        src_path, src_wl = traffic_source(kernel, wl_name, store)
        out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
               "traffic": traffic,
               "kernel": kernel, "kernel_ms": kernel_ms, "bytes_per_lup": kbytes,
               "step_achieved": step_gbs, "step_frac": step_gbs / peak, "step_bytes_per_lup": STEP_BYTES[store],
               "peak_source": f"{peak_src} hbm_gbs"}
        if traffic is not None and src_wl != wl_name:
            out["traffic_source"] = (f"{os.path.relpath(src_path, ROOT)}: ncu DRAM bytes of the same kernel on the "
                                     f"{src_wl} box, scaled per node to this box")
        return out

    peak, peak_src = hbm_peak()

    # ---- device-timed region: K steps of the chosen store -------------------------------------
    sampler = ClockSampler(local)
    ms, kernel_ms, obs, s = device_timed(args.store, args.steps, sampler)
    clocks = sampler.stop()
    ms_max = replica_max(ms, world, "cuda")

    # ---- end to end through the public API from pinned host buffers --------------------------
    phi_h = torch.from_numpy(phi0.reshape(-1)).pin_memory().numpy()
    u_h = torch.from_numpy(u0.reshape(-1)).pin_memory().numpy()
    ps_h = torch.from_numpy(ps0.reshape(-1)).pin_memory().numpy()
    outs = [torch.empty(n, dtype=torch.float32).pin_memory().numpy() for n in (N, 3 * N, N)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init_fields(phi_h, u_h, ps_h)
    s.step(args.steps)
    s.observables(allow_nonfinite=True)
    s.read_fields(*outs)
    e2e_s = replica_max(time.perf_counter() - t0, world, "cuda")
    s.close()

    # ---- the other population stores on the same workload (device-timed, fewer steps) -------
    compare = {}
    if not args.no_store_compare and args.path in (0, 1):
        kc = min(args.steps, 2000)
        for store in STORES:
            if store == args.store:
                continue
            cms, ckms, cobs, cs = device_timed(store, kc)
            cs.close()
            compare[store] = {"value": world * N * kc / (cms * 1e-3) / 1e6, "unit": "MLUPS", "steps": kc,
                              "ms_per_step": cms / kc, "roofline": roofline(store, cms / kc, ckms),
                              "sum_phi_after": cobs["sum_phi"], "nonfinite_after": cobs["n_nonfinite"]}

    # ---- the rising bubble beside the headline workload (device-timed, fewer steps) ----------
    bubble = None
    if args.workload != "rising_bubble" and not args.no_bubble and args.path in (0, 1):
        bw = workload("rising_bubble")
        bf = fields_of(bw)
        bubble = {"workload": bw.name, "nodes": bw.n}
        kb = min(args.steps, 2000)
        for store in ("fp32", "mom_bf16"):
            bms, bkms, bobs, bs = device_timed(store, kb, w=bw, fields=bf)
            bs.close()
            bubble[store] = {"value": world * bw.n * kb / (bms * 1e-3) / 1e6, "unit": "MLUPS", "steps": kb,
                             "ms_per_step": bms / kb,
                             "roofline": roofline(store, bms / kb, bkms, "rising_bubble", bw.n),
                             "sum_phi_after": bobs["sum_phi"], "nonfinite_after": bobs["n_nonfinite"]}
        del bf

    ensemble = None if args.no_ensemble or rank != 0 else run_ensemble(args, stream)
    closure_net = None
    if not args.no_closure and rank == 0:
        from paper_2501_00846_b300 import closure
        closure_net = closure.time_network(64, reps=20, stream=stream)
        closure_net["peak_tflops"] = bf16_peak()
        closure_net["frac"] = closure_net["forward_tflops"] / closure_net["peak_tflops"]

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    value = replica_mlups(N, args.steps, ms_max * 1e-3, world)
    dtype = {"fp32": "f32", "bf16": "f32 compute, bf16 store", "fp16": "f32 compute, f16 store",
             "mom": "f32, moment store", "mom_bf16": "f32 compute, bf16 moment store",
             "mom_fp16": "f32 compute, f16 moment store"}[args.store]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic",
        "config": {"workload": wl.name, "nodes": N, "store": args.store, "path": args.path, "split": args.split,
                   "l2": f"state {STATE_FLOATS[args.store] * 4 * N / 1e9:.2f} GB per copy > 126 MB L2: inputs "
                         "larger than L2, no flush",
                   "parallelism": f"replicas x{world}", "sum_phi_after": obs["sum_phi"],
                   "nonfinite_after": obs["n_nonfinite"]},
        "roofline": roofline(args.store, ms / args.steps, kernel_ms),
        "e2e": {"value": replica_mlups(N, args.steps, e2e_s, world), "unit": "MLUPS",
                "h2d_bytes_per_step": 5 * 4 * N / args.steps,
                "d2h_bytes_per_step": (5 * 4 * N + 8 * 64) / args.steps,
                "includes": "init_fields from pinned host, K steps, observables, read_fields to pinned host"},
        "gpu_launches": args.steps * LAUNCHES_PER_STEP[args.path],
        "clocks": clocks,
    }
    if compare:
        line["store_compare"] = compare
    if bubble is not None:
        line["rising_bubble"] = bubble
    if ensemble is not None:
        line["ensemble"] = ensemble
    if closure_net is not None:
        line["closure_network"] = closure_net
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        v, desc, cores = oracle_sample(args.cpu_seconds, args.workload)
        line["cpu_baseline"] = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc}
        # the same oracle on one thread, on a third of the time
        oracle.set_threads(1)
        try:
            v1, desc1, _ = oracle_sample(max(2.0, args.cpu_seconds / 3), args.workload)
        finally:
            oracle.set_threads(cores)
        line["cpu_baseline"]["single_thread"] = {"value": v1, "unit": "MLUPS", "cores": 1, "sample": desc1}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
