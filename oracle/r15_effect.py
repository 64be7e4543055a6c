"""How far reading R15 moves the FP64 oracle from the printed Allen-Cahn sharpening term.

The paper's sharpening flux is kappa_AC phi (1 - phi) n (Section "Allen-Cahn equation for
interface tracking"); the oracle and the GPU path take the weight as max(phi (1 - phi), 0)
(reading R15), which differs only where phi has left [0, 1].  This script runs the FP64 oracle
both ways from the same seeded inputs and prints, per workload, the largest |delta phi| over the
run and the change of the integral diagnostics at the end.  Test infrastructure like the rest of
oracle/: it imports nothing from the CUDA package except the seeded input generators.

    python -m oracle.r15_effect
"""
import sys

import numpy as np

import oracle
from paper_2501_00846_b300 import inputs

CASES = [
    ("static droplet 48^3 at rest (R = 12, ratio 10), 200 steps", inputs.static_droplet(L=48), 200),
    ("static droplet 48^3 with velocity noise 0.01, 200 steps", inputs.static_droplet(L=48, noise=0.01, seed=1234), 200),
    ("rising bubble 24 x 24 x 96 (R = 6, ratio 100, walls), 800 steps",
     inputs.rising_bubble(nx=24, ny=24, nz=96, R=6.0, zc=16.0, rho_ratio=100.0), 800),
]
KEYS = ("sum_phi", "mass", "p_liq", "p_gas", "centroid_liq", "centroid_gas", "vel_liq", "vel_gas", "phi_min",
        "phi_max")


def run_case(wl, steps, every=20):
    out = {}
    states = []
    for lit in (0, 1):
        P = oracle.Params(literal_weight=lit, **wl.params())
        states.append((P, oracle.init(P, wl.phi0(), wl.u0(), wl.pstar_init())))
    dphi = 0.0
    done = 0
    while done < steps:
        n = min(every, steps - done)
        states = [(P, oracle.run(P, s, n)) for P, s in states]
        done += n
        dphi = max(dphi, float(np.abs(states[0][1].phi - states[1][1].phi).max()))
    (P0, s0), (P1, s1) = states
    o0, o1 = oracle.observables(P0, s0), oracle.observables(P1, s1)
    out["max_dphi"] = dphi
    out["max_du"] = float(np.abs(s0.u - s1.u).max())
    out["umax"] = o0["umax"]
    for k in KEYS:
        a, b = np.atleast_1d(o0[k]), np.atleast_1d(o1[k])
        out[k] = (a.tolist(), (b - a).tolist())
    return out


def main():
    for name, wl, steps in CASES:
        r = run_case(wl, steps)
        print(f"== {name}")
        print(f"   max over the run |phi(R15) - phi(printed)| = {r['max_dphi']:.3e};  "
              f"max |u(R15) - u(printed)| at the end = {r['max_du']:.3e} (max |u| {r['umax']:.3e})")
        for k in KEYS:
            v, d = r[k]
            print(f"   {k:13s} R15 {np.array2string(np.array(v), precision=8)}  printed - R15 "
                  f"{np.array2string(np.array(d), precision=3)}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
