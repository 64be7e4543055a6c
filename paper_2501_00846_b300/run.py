"""Run a named synthetic workload for a number of steps and print its diagnostics as JSON lines.

    python -m paper_2501_00846_b300.run --workload rising_bubble --steps 2000 --every 500
    python -m paper_2501_00846_b300.run --workload droplet256 --storage bf16 --steps 100
    python -m paper_2501_00846_b300.run --workload ensemble32 --steps 100

Workloads: ``rising_bubble`` (128 x 128 x 256, walls on z, density ratio 1000, viscosity ratio
100, Eo = 10, Mo = 1e-4), ``dropletL`` (static droplet in a periodic L^3 box, R = L/4, density
and viscosity ratio 10, sigma = 0.01), ``ensembleN`` (the first N boxes of the batched ensemble of
seeded uneven droplets, inputs.droplet_ensemble, advanced together with the default launch
tuning; diagnostics of every box).  Everything runs on the current CUDA device through the
C ABI; the process fails if the CUDA library is missing.  Also the launch driver of the
committed ncu summaries (a fixed, small number of steps of one workload).
"""
import argparse
import json
import sys

import numpy as np

from . import inputs, solver

STORAGE = {"fp32": solver.LBM_FP32, "bf16": solver.LBM_BF16, "fp16": solver.LBM_FP16, "mom": solver.LBM_MOM,
           "mom_bf16": solver.LBM_MOM_BF16, "mom_fp16": solver.LBM_MOM_FP16}


def workload(name: str):
    if name == "rising_bubble":
        return inputs.rising_bubble()
    if name.startswith("droplet"):
        L = int(name[len("droplet"):])
        return inputs.static_droplet(L=L)
    raise SystemExit(f"unknown workload {name!r}")


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="rising_bubble")
    ap.add_argument("--storage", choices=sorted(STORAGE), default="fp32")
    ap.add_argument("--path", type=int, default=0)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--every", type=int, default=0, help="print diagnostics every this many steps (0: at the end)")
    a = ap.parse_args(argv)

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device")
    torch.cuda.set_device(0)
    if a.workload.startswith("ensemble"):
        return run_ensemble(a)
    wl = workload(a.workload)
    s = solver.from_workload(wl, storage=STORAGE[a.storage])
    try:
        s.set_path(a.path)
        s.set_split(a.split)
        every = a.every if a.every > 0 else max(a.steps, 1)
        done = 0
        while done < a.steps:
            n = min(every, a.steps - done)
            s.step(n)
            done += n
            o = s.observables(allow_nonfinite=True)
            print(json.dumps({"workload": a.workload, "storage": a.storage, "step": done,
                              **{k: (list(v) if isinstance(v, (list, tuple, np.ndarray)) else v)
                                 for k, v in o.items()}}), flush=True)
            if o["n_nonfinite"] > 0:
                return 1
    finally:
        s.close()
    return 0


def run_ensemble(a) -> int:
    """The first N boxes of inputs.droplet_ensemble() in one ensemble; diagnostics of every box."""
    n = int(a.workload[len("ensemble"):])
    wls = inputs.droplet_ensemble()[:n]
    e = solver.ensemble_from_workloads(wls, storage=STORAGE[a.storage])
    try:
        every = a.every if a.every > 0 else max(a.steps, 1)
        done = 0
        while done < a.steps:
            k = min(every, a.steps - done)
            e.step(k)
            done += k
            bad = 0
            for b in range(n):
                o = e.observables(b, allow_nonfinite=True)
                bad += o["n_nonfinite"] > 0
            print(json.dumps({"workload": a.workload, "storage": a.storage, "step": done, "boxes": n,
                              "nodes": int(e.n), "boxes_nonfinite": int(bad)}), flush=True)
            if bad:
                return 1
    finally:
        e.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
