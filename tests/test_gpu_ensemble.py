"""Batched ensemble (lbm_ens_*): every box must evolve exactly as the same box does alone through
lbm_step, for every launch configuration, and the one-box path is itself checked against the FP64
oracle; one ensemble box is also compared with the oracle directly."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    solver.load()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _mixed_boxes():
    """Uneven boxes: cubes of several sizes and properties, a ragged walled bubble with gravity,
    the minimum 4^3 box, a thin box narrower than one Allen–Cahn tile, and a box 128 wide (which
    the one-box path updates with the vector Allen–Cahn kernel, the ensemble with the scalar one:
    the two must give the same bits)."""
    wls = inputs.droplet_ensemble(n=3, seed=7, L_min=24, L_max=40)
    b = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    b.noise, b.seed = 0.005, 99
    wls.append(b)
    wls.append(inputs.static_droplet(L=4, radius=1.5, noise=0.01, seed=3))
    thin = inputs.static_droplet(L=16, radius=4.0, noise=0.01, seed=4)
    thin.nx, thin.ny, thin.nz = 5, 33, 18
    thin.center = (2.0, 16.0, 9.0)
    wls.append(thin)
    wide = inputs.rising_bubble(nx=128, ny=7, nz=10, R=3.0, zc=5.0, sqrt_gR=0.04, mobility=0.1, rho_ratio=100.0)
    wide.center = (127.0, 3.0, 5.0)
    wide.noise, wide.seed = 0.005, 43
    wls.append(wide)
    return wls


def _alone(wl, nsteps):
    with solver.from_workload(wl) as s:
        s.step(nsteps)
        return s.read_fields()


def _ensemble(wls, nsteps, **tuning):
    with solver.ensemble_from_workloads(wls) as e:
        if tuning:
            e.set_tuning(**tuning)
        e.step(nsteps)
        assert e.step_count == nsteps
        return [e.read_fields(b) for b in range(len(wls))], e.tuning


@pytest.fixture(scope="module")
def mixed():
    wls = _mixed_boxes()
    return wls, [_alone(wl, 21) for wl in wls]


def _assert_same(got, ref, label):
    for b, (a, r) in enumerate(zip(got, ref)):
        for name, x, y in zip(("phi", "u", "p"), a, r):
            assert np.array_equal(x, y), f"{label}: box {b} {name} differs (max {np.abs(x - y).max():.3e})"


def test_ensemble_equals_boxes_run_alone(mixed):
    wls, ref = mixed
    got, tun = _ensemble(wls, 21)   # 21 = one graph of 16 steps + 5 direct steps
    assert tun["graph_steps"] == 16
    _assert_same(got, ref, "default tuning")


@pytest.mark.parametrize("tuning", [
    dict(lbm_block=64, ac_rows=2, ac_zlen=8, graph_steps=0),
    dict(lbm_block=256, ac_rows=4, ac_zlen=1, graph_steps=2),
    dict(lbm_block=128, ac_rows=2, ac_zlen=64, graph_steps=4),
], ids=["small", "thin-chunks", "deep-chunks"])
def test_launch_configuration_does_not_change_results(mixed, tuning):
    wls, ref = mixed
    got, tun = _ensemble(wls, 21, **tuning)
    for k, v in tuning.items():
        assert tun[k] == v
    _assert_same(got, ref, str(tuning))


def test_autotune_leaves_the_state_unchanged(mixed):
    wls, ref = mixed
    with solver.ensemble_from_workloads(wls) as e:
        e.step(5)
        t = e.autotune(reps=3)
        e.step(16)
        got = [e.read_fields(b) for b in range(len(wls))]
    assert t["lbm_block"] in (64, 128, 256) and t["ac_rows"] in (2, 4) and t["ac_zlen"] in (8, 16, 32, 64)
    assert t["lbm_us"] > 0 and t["ac_us"] > 0
    print("autotuned:", t)
    _assert_same(got, ref, "after autotune")


def test_ensemble_box_against_the_oracle():
    """One box of a seeded ensemble (density ratio up to 1000) against the FP64 oracle, 60 steps,
    at the FP32 bars of the one-box parity tests."""
    wls = inputs.droplet_ensemble(n=4, seed=11, L_min=24, L_max=28)
    k = int(np.argmax([wl.rho_l / wl.rho_g for wl in wls]))
    with solver.ensemble_from_workloads(wls) as e:
        e.step(60)
        phi, u, p = e.read_fields(k)
        obs = e.observables(k)
    wl = wls[k]
    P = oracle.Params(**wl.params())
    ps = wl.pstar_init()
    ref = oracle.run(P, oracle.init(P, _f32(wl.phi0()).astype(np.float64), _f32(wl.u0()).astype(np.float64),
                                    None if ps is None else _f32(ps).astype(np.float64)), 60)
    pref = oracle.pressure(P, ref)
    dphi = np.abs(phi - ref.phi).max()
    du = np.abs(u - ref.u).max() / np.abs(ref.u).max()
    dp = np.abs(p - pref).max() / np.abs(pref).max()
    print(f"box {k} (ratio {wl.rho_l / wl.rho_g:.0f}): {dphi:.3e} {du:.3e} {dp:.3e}")
    assert dphi <= 1e-5 and du <= 1e-4 and dp <= 1e-4
    assert math.isclose(obs["sum_phi"], oracle.observables(P, ref)["sum_phi"], rel_tol=1e-6)


def test_seeded_ensemble_subset_runs_and_conserves():
    """The first 24 boxes of the 256-droplet ensemble (sizes 32..96, ratios 10..1000): 200 steps,
    every box finite and its sum phi conserved to FP32 round-off."""
    wls = inputs.droplet_ensemble()[:24]
    with solver.ensemble_from_workloads(wls) as e:
        before = [e.observables(b)["sum_phi"] for b in range(len(wls))]
        e.autotune(reps=2)
        e.step(200)
        after = [e.observables(b) for b in range(len(wls))]
    for b, (s0, o) in enumerate(zip(before, after)):
        assert o["n_nonfinite"] == 0
        assert abs(o["sum_phi"] / s0 - 1) < 1e-5, (b, o["sum_phi"], s0)
        assert o["umax"] < 0.1, (b, o["umax"])


def test_ensemble_errors():
    wls = _mixed_boxes()[:2]
    e = solver.Ensemble([wl.params() for wl in wls])
    try:
        with pytest.raises(solver.LbmError) as err:
            e.step(1)
        assert err.value.status == -6                       # a box is not initialised
        with pytest.raises(solver.LbmError) as err:
            e.observables(5)
        assert err.value.status == -1
        with pytest.raises(solver.LbmError) as err:
            e.set_tuning(lbm_block=100)
        assert err.value.status == -1
        with pytest.raises(solver.LbmError) as err:
            e.set_tuning(graph_steps=3)
        assert err.value.status == -1
    finally:
        e.close()
    bad = dict(wls[0].params(), storage=solver.LBM_BF16)
    with pytest.raises(solver.LbmError) as err:
        solver.Ensemble([wls[1].params(), bad])
    assert err.value.status == -1 and "box 1" in str(err.value)


MOM_STORES = [solver.LBM_MOM, solver.LBM_MOM_BF16, solver.LBM_MOM_FP16]


@pytest.mark.parametrize("store", MOM_STORES, ids=["mom", "mom_bf16", "mom_fp16"])
def test_moment_storage_ensemble_equals_boxes_run_alone(mixed, store):
    """With moment storage the ensemble's lattice Boltzmann kernel runs the one-box tiled kernel's
    code on every (box, tile, z chunk) task; the one-box result does not depend on the z chunks,
    so every box matches its run alone bit for bit (direct steps and graph replays)."""
    wls, _ = mixed
    ref = []
    for wl in wls:
        with solver.from_workload(wl, storage=store) as s:
            s.step(21)
            ref.append(s.read_fields())
    with solver.ensemble_from_workloads(wls, storage=store) as e:
        e.step(21)
        got = [e.read_fields(b) for b in range(len(wls))]
        obs = e.observables(0)
    _assert_same(got, ref, f"moment storage {store}")
    with solver.from_workload(wls[0], storage=store) as s:
        s.step(21)
        o1 = s.observables()
    assert obs["sum_pstar"] == o1["sum_pstar"] and obs["sum_phi"] == o1["sum_phi"]


@pytest.mark.parametrize("n_boxes", [2, 64], ids=["chunked", "whole_boxes"])
def test_moment_storage_task_length_does_not_change_the_result(n_boxes):
    """The moment storages' tasks are as long as the task count allows: 2 boxes of 40^3 (too few
    columns: 32-plane chunks) and 64 of them (enough columns for one task per column of a whole
    box).  Either way every box matches its run alone bit for bit (boxes 0 and the last checked)."""
    store = solver.LBM_MOM_BF16
    wls = inputs.droplet_ensemble(n=n_boxes, seed=11, L_min=40, L_max=40)
    with solver.ensemble_from_workloads(wls, storage=store) as e:
        e.step(7)
        got = [e.read_fields(b) for b in (0, n_boxes - 1)]
    ref = []
    for wl in (wls[0], wls[-1]):
        with solver.from_workload(wl, storage=store) as s:
            s.step(7)
            ref.append(s.read_fields())
    _assert_same(got, ref, f"{n_boxes} boxes")


@pytest.mark.parametrize("store", [solver.LBM_FP32, solver.LBM_MOM_BF16], ids=["fp32", "mom_bf16"])
def test_benchmark_ensemble_sampled_boxes_equal_boxes_run_alone(store):
    """The benchmark's ensemble (256 seeded droplets, 80.9M nodes) in the benchmark's launch
    configuration (autotuned, steps replayed from 16-step graphs): sampled boxes (the first, the
    largest, the last) match their runs alone bit for bit after 20 steps."""
    wls = inputs.droplet_ensemble()
    picks = sorted({0, int(np.argmax([wl.n for wl in wls])), len(wls) - 1})
    with solver.ensemble_from_workloads(wls, storage=store) as e:
        e.autotune(reps=1)
        e.step(20)
        got = [e.read_fields(b) for b in picks]
    ref = []
    for b in picks:
        with solver.from_workload(wls[b], storage=store) as s:
            s.step(20)
            ref.append(s.read_fields())
    _assert_same(got, ref, f"benchmark ensemble {store}")


def test_moment_storage_ensemble_rules():
    """Every box of an ensemble has the same storage; the 2x restriction (closure data) needs FP32
    populations."""
    wls = inputs.droplet_ensemble(n=2, seed=3, L_min=24, L_max=32)
    mixed_params = [dict(wls[0].params(), storage=solver.LBM_FP32), dict(wls[1].params(), storage=solver.LBM_MOM)]
    with pytest.raises(solver.LbmError):
        solver.Ensemble(mixed_params)
    big = inputs.static_droplet(L=24, radius=6.0)
    with solver.ensemble_from_workloads([big], storage=solver.LBM_MOM_BF16) as e:
        coarse_params = dict(big.params(), nx=12, ny=12, nz=12)
        with solver.Solver(**coarse_params) as c:
            c.init_fields(np.zeros((12, 12, 12), np.float32), np.zeros((3, 12, 12, 12), np.float32))
            with pytest.raises(solver.LbmError):
                e.restrict_state(0, c)


@pytest.mark.parametrize("store", [solver.LBM_FP32, solver.LBM_MOM_BF16], ids=["fp32", "mom_bf16"])
def test_persistent_step_equals_boxes_run_alone(mixed, store):
    """One persistent cooperative launch per step (Allen–Cahn tasks, grid barrier, lattice
    Boltzmann work) runs the same device functions as the two-launch form: every box matches its
    run alone bit for bit, also with a non-default tuning."""
    wls, ref = mixed
    if store != solver.LBM_FP32:
        ref = []
        for wl in wls:
            with solver.from_workload(wl, storage=store) as s:
                s.step(21)
                ref.append(s.read_fields())
    # the default tuning (13 and 8 steps: direct launches), another tuning, and 4-step graphs of
    # persistent launches (replayed for steps 1-12 and 15-18)
    for tuning in ({}, dict(lbm_block=64, ac_rows=2, ac_zlen=8), dict(graph_steps=4)):
        with solver.ensemble_from_workloads(wls, storage=store) as e:
            if tuning:
                e.set_tuning(**tuning)
            e.set_persistent(True)
            e.step(13)
            e.step(8)
            assert e.step_count == 21
            got = [e.read_fields(b) for b in range(len(wls))]
        _assert_same(got, ref, f"persistent {store} {tuning}")


@pytest.mark.parametrize("graph_steps", [16, 2], ids=["direct", "graph"])
def test_persistent_barrier_expiry_is_reported_and_the_ensemble_recovers(mixed, graph_steps):
    """The grid barrier's waits are bounded.  The test hook keeps CTA 0 from arriving and cuts the
    limit to 2 ms: every wait expires, lbm_ens_step returns LBM_ERR_TIMEOUT, no step is counted and
    the fields are those of the last completed step; with the hook off the ensemble steps on and
    ends exactly where an undisturbed run ends.  With graph_steps = 2 the persistent launches are
    replayed from 2-step graphs, the stalled call's first two included."""
    wls, ref = mixed
    with solver.ensemble_from_workloads(wls) as e:
        if graph_steps != 16:
            e.set_tuning(graph_steps=graph_steps)
        e.set_persistent(True)
        e.step(10)
        before = [e.read_fields(b) for b in range(len(wls))]
        e.test_stall_barrier(True)
        with pytest.raises(solver.LbmError) as err:
            e.step(3)
        assert err.value.status == -5
        assert e.step_count == 10
        _assert_same([e.read_fields(b) for b in range(len(wls))], before, "after the expired step")
        e.test_stall_barrier(False)
        e.step(11)
        assert e.step_count == 21
        got = [e.read_fields(b) for b in range(len(wls))]
    _assert_same(got, ref, "after recovery")
