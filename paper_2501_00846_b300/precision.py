"""Precision study of the storage formats (FP32, BF16, FP16 populations and moments) on long runs.

    python -m paper_2501_00846_b300.precision --bubble-steps 20000 --droplet-L 512 --droplet-steps 2000

* Rising bubble 128 x 128 x 256 (walls on z, density ratio 1000, viscosity ratio 100, Eo = 10,
  Mo = 1e-4): the bubble's rise velocity and centroid every `--every` steps, and the drift of the
  mass (sum rho) and of sum phi, for each storage.
* Static droplet L^3 (R = L/4, density and viscosity ratio 10, sigma = 0.01): the pressure jump
  p_in - p_out against 2 sigma / R_eff and the drifts of mass and sum phi after `--droplet-steps`
  steps, for each storage.

Prints one JSON object; every number comes from the library's FP64 device reductions.
"""
import argparse
import json
import math
import sys
import time

import numpy as np

from . import inputs, solver

STORES = {"fp32": solver.LBM_FP32, "bf16": solver.LBM_BF16, "fp16": solver.LBM_FP16, "mom": solver.LBM_MOM,
          "mom_bf16": solver.LBM_MOM_BF16, "mom_fp16": solver.LBM_MOM_FP16}


def bubble(steps, every, stores):
    wl = inputs.rising_bubble()
    out = {}
    for name in stores:
        t0 = time.perf_counter()
        s = solver.from_workload(wl, storage=STORES[name])
        o0 = s.observables()
        rows = []
        for k in range(every, steps + 1, every):
            s.step(every)
            o = s.observables(allow_nonfinite=True)
            rows.append({"step": k, "z": o["centroid_gas"][2], "w": o["vel_gas"][2], "umax": o["umax"],
                         "nonfinite": o["n_nonfinite"]})
        o = s.observables(allow_nonfinite=True)
        s.close()
        out[name] = {"trace": rows, "mass_drift": o["mass"] / o0["mass"] - 1.0,
                     "sum_phi_drift": o["sum_phi"] / o0["sum_phi"] - 1.0, "seconds": time.perf_counter() - t0}
    ref = out["fp32"]["trace"] if "fp32" in out else None
    for name in out:
        if ref is not None and name != "fp32":
            out[name]["w_rel_diff_final"] = out[name]["trace"][-1]["w"] / ref[-1]["w"] - 1.0
            out[name]["z_diff_final"] = out[name]["trace"][-1]["z"] - ref[-1]["z"]
    return out


def droplet(L, steps, stores):
    wl = inputs.static_droplet(L=L)
    phi0 = np.ascontiguousarray(wl.phi0(), np.float32)
    u0 = np.ascontiguousarray(wl.u0(), np.float32)
    ps0 = np.ascontiguousarray(wl.pstar_init(), np.float32)
    out = {}
    for name in stores:
        t0 = time.perf_counter()
        s = solver.Solver(storage=STORES[name], **wl.params())
        s.init_fields(phi0, u0, ps0)
        o0 = s.observables()
        s.step(steps)
        o = s.observables(allow_nonfinite=True)
        s.close()
        reff = (3.0 * o["sum_phi"] / (4.0 * math.pi)) ** (1.0 / 3.0)
        dp = o["p_liq"] - o["p_gas"]
        out[name] = {"dp": dp, "laplace_ratio": dp / (2.0 * wl.sigma / reff), "mass_drift": o["mass"] / o0["mass"] - 1.0,
                     "sum_phi_drift": o["sum_phi"] / o0["sum_phi"] - 1.0, "umax": o["umax"],
                     "nonfinite": o["n_nonfinite"], "seconds": time.perf_counter() - t0}
    if "fp32" in out:
        for name in out:
            if name != "fp32":
                out[name]["dp_rel_diff"] = out[name]["dp"] / out["fp32"]["dp"] - 1.0
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--bubble-steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--droplet-L", type=int, default=512)
    ap.add_argument("--droplet-steps", type=int, default=2000)
    ap.add_argument("--stores", default="fp32,bf16,fp16,mom,mom_bf16,mom_fp16")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    stores = a.stores.split(",")
    res = {"bubble": bubble(a.bubble_steps, a.every, stores) if a.bubble_steps > 0 else None,
           "droplet": droplet(a.droplet_L, a.droplet_steps, stores) if a.droplet_steps > 0 else None,
           "config": vars(a)}
    print(json.dumps(res))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
