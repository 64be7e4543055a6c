"""Learned closure: training data from the solver's own fine-grid runs, training with the library's
network kernels, and evaluation against the fine solver.

The closure corrects (phi, ubar) of a 2x-coarser grid once every `every` coarse steps (default 8).
Data: seeded head-on droplet collisions (inputs.collision_set) run on the fine grid (L^3) in
batches through the ensemble; at each snapshot the fine state is restricted 2x into a coarse
context (populations, phi and ubar averaged over the 8 fine nodes of a coarse cell), the coarse
context takes `every` steps (= 2 x every fine steps in acoustic scaling) while the fine batch takes
twice as many, and the pair

    x = features(coarse state after those steps),    t = (restricted fine (phi, u) - coarse (phi, ubar)) / out_scale

is stored on the device.  Training: Adam on the mean-squared error, minibatches accumulated in
the network's gradient buffer.  Evaluation: a held-out collision run three ways from the same
restricted initial state -- the fine solver (restricted 2x, the reference), the plain coarse solver,
and the coarse solver corrected by the network after every `every` steps -- with RMS errors of phi
and u against that reference and device times of each.  Trained on one-step defects, the velocity
correction drives the closed loop away from its data and is applied with a factor (--u-relax);
trained on 8-step defects, the network's own velocity prediction lowers the u error.

Everything numerical runs in the library's CUDA kernels; torch provides device memory and the
stream.

    python -m paper_2501_00846_b300.closure --traj 200 --epochs 6 --out closure_run.json
"""
import argparse
import json
import math
import sys
import time

import numpy as np

from . import inputs, solver


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _coarse_context(col, stream):
    """A coarse context with the collision's coarse parameters (state set later by restriction)."""
    p = col.coarse_params()
    s = solver.Solver(stream=stream, **p)
    n = p["nx"] * p["ny"] * p["nz"]
    s.init_fields(np.zeros(n, np.float32), np.zeros(3 * n, np.float32))
    return s


IDENTITY = solver.LbmClosureNorm.make([0.0] * 5, [1.0] * 5, [1.0] * 4)


def generate(collisions, snapshots=20, stride=48, batch=25, norm=IDENTITY, stream=None, log=None, every=1,
             burn=(0, 0), seed=0, policy=None, rollout=1):
    """Training pairs (X [S, 5, Nc], T [S, 4, Nc], device tensors) from len(collisions) fine runs,
    one snapshot every `stride` fine steps.

    At a snapshot the fine state is restricted into a coarse context, which then runs `rollout`
    legs; a leg is b + `every` coarse steps (b drawn per snapshot from the range `burn`, seeded)
    while the fine run takes twice as many, and gives the pair
        x = features(coarse state after the leg),
        t = (restricted fine (phi, u) - coarse (phi, ubar)) / out_scale.
    With a `policy` (network, norm), the coarse state is corrected by that network after every
    leg but the last, so the later legs start from states the corrected solver itself reaches
    (on-policy data for iterated training); without one, rollout must be 1.  Returns
    len(collisions) * snapshots * rollout pairs."""
    import torch
    if policy is None and rollout != 1:
        raise ValueError("rollouts longer than one leg need a policy network")
    stream = stream or torch.cuda.current_stream()
    L = collisions[0].L
    Nc = (L // 2) ** 3
    S = len(collisions) * snapshots * rollout
    X = torch.empty((S, 5, Nc), device="cuda")
    T = torch.empty((S, 4, Nc), device="cuda")
    ref = torch.empty(4 * Nc, device="cuda")
    idx = 0
    rng = np.random.default_rng(seed)
    burns = [int(rng.integers(burn[0], burn[1] + 1)) for _ in range(snapshots)]
    if stride < 2 * rollout * (max(burns) + every):
        raise ValueError("stride too short for the rollout")
    with torch.cuda.stream(stream):
        for b0 in range(0, len(collisions), batch):
            cols = collisions[b0:b0 + batch]
            t0 = time.perf_counter()
            ens = solver.Ensemble([c.params() for c in cols], stream=stream)
            for k, c in enumerate(cols):
                phi, u, ps = c.fields()
                ens.init_fields(k, _f32(phi), _f32(u), _f32(ps))
            coarse = [_coarse_context(c, stream) for c in cols]
            restricted = _coarse_context(cols[0], stream)
            for snap in range(snapshots):
                m = burns[snap] + every
                ens.step(stride - 2 * m * rollout)
                for k in range(len(cols)):
                    ens.restrict_state(k, coarse[k])
                for leg in range(rollout):
                    ens.step(2 * m)
                    for k in range(len(cols)):
                        coarse[k].step(m)
                        ens.restrict_state(k, restricted)
                        restricted.read_fields(phi=ref[:Nc], u=ref[Nc:])
                        solver.closure_features(coarse[k], norm, X[idx].reshape(-1))
                        solver.closure_target(coarse[k], ref, norm, T[idx].reshape(-1))
                        idx += 1
                        if policy is not None and leg < rollout - 1:
                            solver.closure_apply(coarse[k], policy[0], policy[1])
            torch.cuda.synchronize()
            for c in coarse:
                c.close()
            restricted.close()
            ens.close()
            if log:
                log(f"data: collisions {b0}..{b0 + len(cols) - 1}, {idx} pairs, {time.perf_counter() - t0:.1f} s")
    return X[:idx], T[:idx]


def estimate_norm(collisions, snapshots=6, stride=48, stream=None, every=1):
    """Input shifts and scales (mean and standard deviation of phi, u, p) and output scales
    (standard deviation of the raw corrections) from a small pilot set, on the host."""
    X, T = generate(collisions, snapshots=snapshots, stride=stride, batch=len(collisions), stream=stream, every=every)
    x = X.permute(1, 0, 2).reshape(5, -1).double().cpu().numpy()
    t = T.permute(1, 0, 2).reshape(4, -1).double().cpu().numpy()
    shift = x.mean(axis=1)
    scale = np.maximum(x.std(axis=1), 1e-12)
    shift[0], scale[0] = 0.5, 0.5                      # phi in [0, 1]
    shift[1:4] = 0.0                                   # velocities: symmetric
    out = np.maximum(t.std(axis=1), 1e-12)
    return solver.LbmClosureNorm.make(shift, scale, out)


def train(net, X, T, epochs=4, lr=1e-3, batch=4, seed=0, log=None):
    """Adam over the pairs in random order, `batch` samples per step; cosine learning-rate decay.
    X, T: tensors [S, ...] or lists of them (several data sets used together without copying).
    Returns the mean loss of every epoch."""
    if isinstance(X, (list, tuple)):
        where = [(j, i) for j, x in enumerate(X) for i in range(x.shape[0])]
        Xl, Tl = X, T
    else:
        where = [(0, i) for i in range(X.shape[0])]
        Xl, Tl = [X], [T]
    S = len(where)
    rng = np.random.default_rng(seed)
    steps = epochs * math.ceil(S / batch)
    k = 0
    history = []
    for ep in range(epochs):
        order = rng.permutation(S)
        tot = 0.0
        t0 = time.perf_counter()
        for i in range(0, S, batch):
            ids = order[i:i + batch]
            for j, s in enumerate(ids):
                d, i_ = where[int(s)]
                tot += net.grad(Xl[d][i_].reshape(-1), Tl[d][i_].reshape(-1), accumulate=j > 0)
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * k / steps))
            net.adam_step(rate, 1.0 / len(ids))
            k += 1
        history.append(tot / S)
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4e} ({time.perf_counter() - t0:.1f} s)")
    return history


def evaluate(net, norm, col, coarse_steps=240, every=24, stream=None, apply_every=1):
    """RMS errors of phi and u of the plain and the corrected coarse runs against the restricted
    fine run of collision `col` (checked every `every` coarse steps), and device times per coarse
    step of the three runs.  The correction is applied after every `apply_every` coarse steps."""
    import torch
    stream = stream or torch.cuda.current_stream()
    n = (col.L // 2) ** 3
    out = {"checkpoints": [], "steps": coarse_steps}
    with torch.cuda.stream(stream):
        fine = solver.Ensemble([col.params()], stream=stream)
        phi, u, ps = col.fields()
        fine.init_fields(0, _f32(phi), _f32(u), _f32(ps))
        plain, corr, restricted = (_coarse_context(col, stream) for _ in range(3))
        fine.restrict_state(0, plain)
        fine.restrict_state(0, corr)
        e_plain, e_corr = [], []
        for k in range(1, coarse_steps + 1):
            fine.step(2)
            plain.step(1)
            corr.step(1)
            if k % apply_every == 0:
                solver.closure_apply(corr, net, norm)
            if k % every == 0:
                fine.restrict_state(0, restricted)
                jp, ju, _ = restricted.read_fields()
                row = {"step": k}
                for name, s, acc in (("plain", plain, e_plain), ("closure", corr, e_corr)):
                    sp, su, _ = s.read_fields()
                    ephi = float(np.sqrt(np.mean((sp.astype(np.float64) - jp) ** 2)))
                    eu = float(np.sqrt(np.mean((su.astype(np.float64) - ju) ** 2)))
                    row[name] = {"phi_rms": ephi, "u_rms": eu}
                    acc.append((ephi, eu))
                out["checkpoints"].append(row)
        for name, acc in (("plain", e_plain), ("closure", e_corr)):
            a = np.array(acc)
            out[name] = {"phi_rms_mean": float(a[:, 0].mean()), "u_rms_mean": float(a[:, 1].mean())}
        out["ratio_phi"] = out["closure"]["phi_rms_mean"] / out["plain"]["phi_rms_mean"]
        out["ratio_u"] = out["closure"]["u_rms_mean"] / out["plain"]["u_rms_mean"]
        # device time per coarse step of each run (same number of steps, after the error run)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        nrep = 50

        def timed(fn):
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(nrep):
                fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / nrep

        ref_fine = solver.Solver(stream=stream, **col.params())    # the one-box fine path, for timing
        ref_fine.init_fields(_f32(phi), _f32(u), _f32(ps))
        out["ms_per_coarse_step"] = {
            "fine_2_steps": timed(lambda: ref_fine.step(2)),
            "coarse": timed(lambda: plain.step(1)),
            "coarse_with_closure": timed(lambda: (corr.step(apply_every), solver.closure_apply(corr, net, norm)))
            / apply_every,
        }
        out["apply_every"] = apply_every
        for s in (plain, corr, restricted, ref_fine):
            s.close()
        fine.close()
    out["nodes"] = {"fine": col.L ** 3, "coarse": n}
    return out


# Checks of a corrected coarse state (coarse lattice units): no non-finite value, phi inside
# [phi_min, phi_max], max |u| below umax (far below the lattice speed of sound), and sum phi within
# a relative sum_phi_drift of the start (the correction conserves it; a drift means trouble).
DEFAULT_LIMITS = {"phi_min": -0.1, "phi_max": 1.1, "umax": 0.2, "sum_phi_drift": 1e-3}


def failed_checks(obs, obs0, limits=None):
    """Reasons why the state with observables obs fails the checks (empty when it passes); obs0:
    the observables of the run's first state."""
    lim = dict(DEFAULT_LIMITS, **(limits or {}))
    bad = []
    if obs["n_nonfinite"] > 0:
        bad.append(f"{obs['n_nonfinite']:.0f} non-finite nodes")
        return bad
    if obs["phi_min"] < lim["phi_min"] or obs["phi_max"] > lim["phi_max"]:
        bad.append(f"phi in [{obs['phi_min']:.4f}, {obs['phi_max']:.4f}]")
    if obs["umax"] > lim["umax"]:
        bad.append(f"max |u| {obs['umax']:.4f}")
    if abs(obs["sum_phi"] - obs0["sum_phi"]) > lim["sum_phi_drift"] * abs(obs0["sum_phi"]):
        bad.append(f"sum phi drifted by {obs['sum_phi'] / obs0['sum_phi'] - 1:.2e}")
    return bad


def run_with_fallback(net, norm, col, coarse_steps=240, check_every=24, apply_every=8, limits=None, stream=None):
    """The corrected coarse run of collision `col`, with the plain fine solver as its fallback.

    The run starts from the collision's fine initial state restricted 2x and applies the network
    after every `apply_every` coarse steps.  Every `check_every` coarse steps (and at the end) the
    state is checked (failed_checks); a state that passes is kept on the device as the checkpoint.
    When a check fails, the run returns to the last checkpoint, prolongs it 2x to the fine grid
    (lbm_prolong2_state) and finishes the remaining time with the plain fine solver, two fine steps
    per coarse step.  Returns (record, solver): the record holds every check and, after a
    fallback, the step it was detected at and the step the fine run restarted from; the solver is
    the context holding the final state (the coarse one, or the fine one after a fallback), owned
    by the caller."""
    import torch
    stream = stream or torch.cuda.current_stream()
    L = solver.load()
    with torch.cuda.stream(stream):
        ens = solver.Ensemble([col.params()], stream=stream)
        phi, u, ps = col.fields()
        ens.init_fields(0, _f32(phi), _f32(u), _f32(ps))
        corr = _coarse_context(col, stream)
        ens.restrict_state(0, corr)
        ens.close()
        n = corr.n
        ck = (torch.empty(27 * n, device="cuda"), torch.empty(n, device="cuda"), torch.empty(3 * n, device="cuda"))

        def checkpoint():
            solver._check(L.lbm_get_state(corr._ctx, ck[0].data_ptr(), ck[1].data_ptr(), ck[2].data_ptr(), 1))

        record = {"checks": [], "fallback": None, "final": "coarse", "coarse_steps": coarse_steps}
        fine = None
        try:
            checkpoint()
            ck_step = 0
            obs0 = corr.observables(allow_nonfinite=True)
            for k in range(1, coarse_steps + 1):
                corr.step(1)
                if k % apply_every == 0:
                    solver.closure_apply(corr, net, norm)
                if k % check_every and k != coarse_steps:
                    continue
                bad = failed_checks(corr.observables(allow_nonfinite=True), obs0, limits)
                record["checks"].append({"step": k, "failed": bad})
                if not bad:
                    checkpoint()
                    ck_step = k
                    continue
                # fallback: the last checkpoint, prolonged to the fine grid, finishes the run
                corr.set_state(*ck, step=ck_step)
                fine = solver.Solver(stream=stream, **col.params())
                fine.init_fields(np.zeros(fine.n, np.float32), np.zeros(3 * fine.n, np.float32))
                solver.prolong2_state(corr, fine)
                fine.step(2 * (coarse_steps - ck_step))
                record["fallback"] = {"detected_at": k, "restart_from": ck_step,
                                      "fine_steps": 2 * (coarse_steps - ck_step)}
                record["final"] = "fine"
                corr.close()
                return record, fine
        except BaseException:
            corr.close()
            if fine is not None:
                fine.close()
            raise
    return record, corr


def _block_mean(a, f):
    """Mean over f x f x f blocks of the last three axes."""
    *lead, nz, ny, nx = a.shape
    return a.reshape(*lead, nz // f, f, ny // f, f, nx // f, f).mean(axis=(-5, -3, -1))


def accuracy_ladder(net, norm, col, coarse_steps=240, check_every=24, resolutions=(64, 96), compare=32,
                    stream=None, apply_every=1):
    """Accuracy and cost of the plain solver on a ladder of grids against the fine run, beside the
    corrected coarse run.  The fine collision col (col.L^3) is the reference; every other run is
    the same physical collision rescaled to its grid (inputs.rescaled_collision: acoustic
    scaling, the initial profiles of the same physical width, the solver's interface width W
    lattice units everywhere), started from its own initial fields.  Each run is compared at the
    same physical times, every check_every steps of the coarsest grid, after block-averaging phi
    and u to compare^3 (every grid a multiple of it).  The corrected run is the coarsest grid
    (col.L / 2) with the closure applied every apply_every steps.  Returns per grid the mean RMS
    error of phi and u over the checks and the device milliseconds per unit physical time (one
    step of the coarsest grid), plus the corrected run's."""
    import torch
    stream = stream or torch.cuda.current_stream()
    Lc = col.L // 2
    assert all(L % compare == 0 for L in resolutions + (col.L,)) and Lc in resolutions
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"compare": f"{compare}^3", "coarse_steps": coarse_steps, "runs": {}}
    with torch.cuda.stream(stream):
        def make(L):
            c = col if L == col.L else inputs.rescaled_collision(col, L)
            s = solver.Solver(stream=stream, **c.params())
            phi, u, ps = c.fields()
            s.init_fields(_f32(phi), _f32(u), _f32(ps))
            return s

        # steps of each grid per coarse step: L / Lc (acoustic scaling), integral for every grid
        runs = {("fine", col.L): make(col.L)}
        for L in resolutions:
            runs[("plain", L)] = make(L)
        runs[("closure", Lc)] = make(Lc)
        per = {k: k[1] // Lc if k[1] % Lc == 0 else None for k in runs}
        for k in runs:
            if per[k] is None:
                per[k] = k[1] / Lc
        errs = {k: [] for k in runs if k[0] != "fine"}
        done = {k: 0 for k in runs}
        for c in range(1, coarse_steps // check_every + 1):
            target = c * check_every
            for k, s in runs.items():
                n = int(round(target * per[k])) - done[k]
                if k[0] == "closure":
                    for _ in range(n):
                        s.step(1)
                        done[k] += 1
                        if done[k] % apply_every == 0:
                            solver.closure_apply(s, net, norm)
                else:
                    s.step(n)
                    done[k] += n
            ref = runs[("fine", col.L)].read_fields()
            rphi = _block_mean(ref[0].astype(np.float64), col.L // compare)
            ru = _block_mean(ref[1].astype(np.float64), col.L // compare)
            for k in errs:
                f = runs[k].read_fields()
                phi = _block_mean(f[0].astype(np.float64), k[1] // compare)
                u = _block_mean(f[1].astype(np.float64), k[1] // compare)
                errs[k].append((float(np.sqrt(np.mean((phi - rphi) ** 2))), float(np.sqrt(np.mean((u - ru) ** 2)))))

        def timed(k, nrep=20):
            s = runs[k]
            steps = per[k]
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(nrep):
                if k[0] == "closure":
                    s.step(1)
                    if (done[k] + 1) % apply_every == 0:
                        solver.closure_apply(s, net, norm)
                    done[k] += 1
                else:
                    s.step(int(round(steps)) if float(steps).is_integer() else 1)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / nrep
            return ms if float(steps).is_integer() or k[0] == "closure" else ms * steps

        for k in runs:
            e = np.array(errs[k]) if k in errs else None
            out["runs"][f"{k[0]}_{k[1]}"] = {
                "grid": f"{k[1]}^3", "steps_per_coarse_step": per[k], "ms_per_coarse_step": timed(k),
                **({"phi_rms_mean": float(e[:, 0].mean()), "u_rms_mean": float(e[:, 1].mean())} if e is not None else {})}
        for s in runs.values():
            s.close()
    return out


def equal_accuracy(ladder, coarse=64, finer=96):
    """From an accuracy ladder: fit the plain solver's phi error to e(L) = C L^-p through the two
    plain grids, solve e(L*) = the corrected run's error, and price the plain solver at L* with
    the cost law t(L) = t(coarse) (L / coarse)^q fitted through the same two grids' measured
    times.  Returns L*, the plain solver's time per unit physical time at L*, and the corrected
    run's."""
    r = ladder["runs"]
    e1, e2 = r[f"plain_{coarse}"]["phi_rms_mean"], r[f"plain_{finer}"]["phi_rms_mean"]
    t1, t2 = r[f"plain_{coarse}"]["ms_per_coarse_step"], r[f"plain_{finer}"]["ms_per_coarse_step"]
    ec, tc = r[f"closure_{coarse}"]["phi_rms_mean"], r[f"closure_{coarse}"]["ms_per_coarse_step"]
    p = math.log(e1 / e2) / math.log(finer / coarse)
    q = math.log(t2 / t1) / math.log(finer / coarse)
    Ls = coarse * (e1 / ec) ** (1.0 / p)
    return {"error_exponent": p, "cost_exponent": q, "equal_accuracy_grid": Ls,
            "plain_ms_at_equal_accuracy": t1 * (Ls / coarse) ** q, "closure_ms": tc,
            "speedup": t1 * (Ls / coarse) ** q / tc}


# useful multiply-adds per node of one forward pass: 27 offsets x (5x32 + 32x32 + 32x32 + 32x4)
FORWARD_MACS_PER_NODE = 27 * sum(o * i for o, i in solver.CNN_LAYERS)


def time_network(L=64, reps=50, kernel=0, seed=3, stream=None):
    """Device time of one forward pass and of one training step (forward, loss, backward) of the
    network on an L^3 grid with seeded inputs, CUDA events over `reps` calls each after a warm-up.
    Returns a dict with milliseconds and the forward pass's useful TFLOP/s (2 flops per
    multiply-add of the unpadded channels)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    with torch.cuda.stream(stream), solver.Network(L, L, L, seed=seed, stream=stream) as net:
        net.set_conv_kernel(kernel)
        g = torch.Generator(device="cuda").manual_seed(seed)
        x = torch.randn(5 * net.n, device="cuda", generator=g)
        t = 0.1 * torch.randn(4 * net.n, device="cuda", generator=g)
        y = torch.empty(4 * net.n, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            ev[0].record(stream)
            for _ in range(reps):
                fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / reps

        fwd = timed(lambda: net.forward(x, y))
        grad = timed(lambda: net.grad(x, t))
        n = net.n
    return {"grid": f"{L}^3", "kernel": kernel, "forward_ms": fwd, "train_step_ms": grad,
            "forward_tflops": 2.0 * FORWARD_MACS_PER_NODE * n / (fwd * 1e-3) / 1e12}


def main(argv=None):
    ap = argparse.ArgumentParser(description="train and evaluate the learned closure")
    ap.add_argument("--traj", type=int, default=200)
    ap.add_argument("--snapshots", type=int, default=20)
    ap.add_argument("--stride", type=int, default=48)
    ap.add_argument("--batch-traj", type=int, default=25)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval", type=int, default=2, help="held-out collisions to evaluate")
    ap.add_argument("--eval-steps", type=int, default=240)
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=None, help="JSON file for the results")
    ap.add_argument("--weights", default=None, help="npz file for the trained parameters and normalisation")
    ap.add_argument("--load", default=None, help="evaluate parameters from an npz written by --weights (no training)")
    ap.add_argument("--phi-only", action="store_true", help="apply only the phi correction when evaluating")
    ap.add_argument("--every", type=int, default=8,
                    help="coarse steps per correction (the network is trained on the defect of this many steps)")
    ap.add_argument("--u-relax", type=float, default=1.0,
                    help="factor on the applied velocity correction (1: the network's own prediction; "
                         "0: the phi correction alone)")
    ap.add_argument("--time-network", type=int, default=0, metavar="L",
                    help="only time the network's forward pass and training step on an L^3 grid")
    ap.add_argument("--ladder", action="store_true",
                    help="also run the accuracy ladder (plain L/2 and 3L/4 grids, corrected L/2) on the "
                         "first held-out collision and report the plain grid of equal phi accuracy")
    ap.add_argument("--policy-rounds", type=int, default=0,
                    help="rounds of on-policy data: roll the coarse run out with the current network, add "
                         "the pairs, retrain")
    ap.add_argument("--rollout", type=int, default=6, help="legs of each on-policy rollout")
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--fallback", action="store_true",
                    help="also run each held-out collision with the fine solver as fallback (run_with_fallback) "
                         "and report its checks")
    a = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    if a.time_network:
        print(json.dumps(time_network(a.time_network, reps=a.reps)))
        return 0
    log = lambda m: print(m, file=sys.stderr, flush=True)
    cols = inputs.collision_set(a.traj + a.eval, seed=a.seed, L=a.L, R=a.L * 20.0 / 128.0)
    train_cols, eval_cols = cols[:a.traj], cols[a.traj:]
    if a.load:
        z = np.load(a.load)
        out_scale = np.array(z["out_scale"], np.float64)
        out_scale[1:] *= 0.0 if a.phi_only else a.u_relax
        norm = solver.LbmClosureNorm.make(z["in_shift"], z["in_scale"], out_scale)
        net = solver.Network(a.L // 2, a.L // 2, a.L // 2, seed=a.seed)
        net.set_params(z["params"])
        res = {"eval": [evaluate(net, norm, c, coarse_steps=a.eval_steps, apply_every=a.every) for c in eval_cols],
               "every": a.every, "u_relax": a.u_relax}
        if a.fallback:
            res["fallback"] = []
            for c in eval_cols:
                record, final = run_with_fallback(net, norm, c, coarse_steps=a.eval_steps, apply_every=a.every)
                final.close()
                res["fallback"].append(record)
        if a.ladder:
            res["ladder"] = accuracy_ladder(net, norm, eval_cols[0], coarse_steps=a.eval_steps,
                                            resolutions=(a.L // 2, 3 * a.L // 4), compare=a.L // 4,
                                            apply_every=a.every)
            res["equal_accuracy"] = equal_accuracy(res["ladder"], coarse=a.L // 2, finer=3 * a.L // 4)
        print(json.dumps(res))
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh, indent=1)
        net.close()
        return 0
    t0 = time.perf_counter()
    norm = estimate_norm(train_cols[:4], stride=a.stride, every=a.every)
    log(f"norm: in_shift {list(norm.in_shift)} in_scale {list(norm.in_scale)} out_scale {list(norm.out_scale)}")
    X, T = generate(train_cols, snapshots=a.snapshots, stride=a.stride, batch=a.batch_traj, norm=norm, log=log,
                    every=a.every)
    t_data = time.perf_counter() - t0
    net = solver.Network(a.L // 2, a.L // 2, a.L // 2, seed=a.seed)
    t1 = time.perf_counter()
    hist = train(net, X, T, epochs=a.epochs, lr=a.lr, log=log)
    applied = solver.LbmClosureNorm.make(norm.in_shift, norm.in_scale,
                                         [norm.out_scale[0]] + [a.u_relax * v for v in list(norm.out_scale)[1:]])
    Xs, Ts = [X], [T]
    for r in range(a.policy_rounds):   # on-policy data from the current network's own rollouts
        # as many pairs per round as the first data set: snapshots / rollout rollouts per collision
        Xp, Tp = generate(train_cols, snapshots=max(1, a.snapshots // a.rollout), stride=a.stride,
                          batch=a.batch_traj, norm=norm,
                          log=log, every=a.every, policy=(net, applied), rollout=a.rollout, seed=r + 1)
        Xs.append(Xp)
        Ts.append(Tp)
        hist += train(net, Xs, Ts, epochs=a.epochs, lr=a.lr, seed=r + 1, log=log)
    t_train = time.perf_counter() - t1
    npairs = sum(x.shape[0] for x in Xs)
    del X, T, Xs, Ts
    evals = [evaluate(net, applied, c, coarse_steps=a.eval_steps, apply_every=a.every) for c in eval_cols]
    res = {"trajectories": a.traj, "pairs": npairs, "epochs": a.epochs, "every": a.every,
           "policy_rounds": a.policy_rounds, "u_relax": a.u_relax, "loss": hist,
           "seconds": {"data": t_data, "train": t_train}, "eval": evals,
           "norm": {"in_shift": list(norm.in_shift), "in_scale": list(norm.in_scale),
                    "out_scale": list(norm.out_scale)}}
    if a.ladder:
        lad = accuracy_ladder(net, applied, eval_cols[0], coarse_steps=a.eval_steps,
                              resolutions=(a.L // 2, 3 * a.L // 4), compare=a.L // 4, apply_every=a.every)
        res["ladder"] = lad
        res["equal_accuracy"] = equal_accuracy(lad, coarse=a.L // 2, finer=3 * a.L // 4)
    print(json.dumps(res))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    if a.weights:
        np.savez(a.weights, params=net.get_params(), in_shift=np.array(norm.in_shift),
                 in_scale=np.array(norm.in_scale), out_scale=np.array(norm.out_scale))
    net.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
