"""Moment-only storage (LBM_MOM, and LBM_MOM_BF16 / LBM_MOM_FP16 with a and B in 16 bits) against
the FP64 oracle, the FP32 population form, and itself.

The moment form keeps (p*, u, a, B) per node in FP32 and rebuilds every streamed population from
them with FP32 arithmetic; it computes the same step as the FP32 population form up to rounding,
so it is held to the FP32 bars: max|d phi| <= 1e-5, relative u and p <= 1e-4 after 100 steps,
integral observables within 0.5% on long runs.  The tiled kernel (path 0) gives identical bits
for every z split (each chunk rebuilds its halo planes' populations with the same arithmetic as
their owners).  It and the one-node-per-thread kernel (path 1) rebuild identical populations, but
the compiler may contract the collision's FP32 products differently in the two kernels, so they
agree to FP32 rounding, not bit for bit.

The 16-bit moment stores round a and B (the non-equilibrium part of the state) once per step.
The oracle emulates exactly that rounding (oracle.Params storage16 = 3 BF16, 4 FP16, pinned against
the representation's moment identities and independent rounding routines in
test_oracle_storage16.py), so each case's bar is derived, as for the 16-bit population stores:
eps16 = |oracle with 16-bit moments - oracle| (max|d phi|, relative du, relative dp), and a GPU run
must lie within FP32 bar + 3 eps16 of the plain oracle (a GPU run is another realisation of the
rounding, so its distance from the plain oracle is of the size of eps16, not below it).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu

MOM = solver.LBM_MOM
STORES = [solver.LBM_MOM, solver.LBM_MOM_BF16, solver.LBM_MOM_FP16]
STORE_IDS = ["f32", "bf16", "fp16"]
FP32_BAR = (1e-5, 1e-4, 1e-4)   # the FP32 bars against the oracle: max|d phi|, rel du, rel dp
SPREAD = 3.0                    # 16-bit stores: bar = FP32 bar + SPREAD eps16
EMULATION = {solver.LBM_MOM_BF16: 3, solver.LBM_MOM_FP16: 4}   # oracle.Params.storage16 of each store


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    solver.load()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _pstar0(wl):
    ps = wl.pstar_init()
    return None if ps is None else _f32(ps)


def _run(wl, nsteps, storage=MOM, path=0, split=0):
    with solver.Solver(storage=storage, **wl.params()) as s:
        s.set_path(path)
        s.set_split(split)
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(nsteps)
        phi, u, p = s.read_fields()
        g, _, _ = s.get_state()
        obs = s.observables()
    return phi, u, p, g, obs


def _oracle(wl, nsteps, storage16=0):
    P = oracle.Params(**wl.params(), storage16=storage16)
    ps = _pstar0(wl)
    st = oracle.run(P, oracle.init(P, _f32(wl.phi0()).astype(np.float64), _f32(wl.u0()).astype(np.float64),
                                   None if ps is None else ps.astype(np.float64)), nsteps)
    return P, st


def _errs(fields, P, ref, u_scale=None):
    """max|d phi|, max|d u| / (u_scale or max|u_ref|), max|d p| / max|p_ref| of fields (phi, u, p)."""
    phi, u, p = fields[:3]
    pref = oracle.pressure(P, ref)
    us = u_scale if u_scale else np.abs(ref.u).max()
    return (float(np.abs(phi - ref.phi).max()), float(np.abs(u - ref.u).max() / us),
            float(np.abs(p - pref).max() / np.abs(pref).max()))


def _eps16(wl, nsteps, store, P, ref, u_scale=None):
    """The 16-bit moment store's own effect on this case: the emulating oracle's distance from the
    plain one (zero for FP32 moments)."""
    if store not in EMULATION:
        return (0.0, 0.0, 0.0)
    P16, ref16 = _oracle(wl, nsteps, EMULATION[store])
    return _errs((ref16.phi, ref16.u, oracle.pressure(P16, ref16)), P, ref, u_scale)


def _bars(wl, nsteps, store, P, ref, factor=1.0, u_scale=None):
    eps = _eps16(wl, nsteps, store, P, ref, u_scale)
    return tuple(factor * FP32_BAR[j] + SPREAD * eps[j] for j in range(3))


def _check(out, P, ref, bars, label, store=MOM, u_scale=None):
    d = _errs(out, P, ref, u_scale)
    print(f"{label} store={store}: max|dphi| {d[0]:.3e} rel du {d[1]:.3e} rel dp {d[2]:.3e}; bars {bars[0]:.3e} "
          f"{bars[1]:.3e} {bars[2]:.3e}")
    assert all(d[j] <= bars[j] for j in range(3)), (label, d, bars)


def _same(a, b):
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)


@pytest.fixture(scope="module")
def droplet48():
    wl = inputs.static_droplet(L=48, radius=12.0, noise=0.01, seed=1234)
    P, ref = _oracle(wl, 100)
    return wl, P, ref, {st: _bars(wl, 100, st, P, ref) for st in STORES}


PATHS = [0, 1]
PATH_IDS = ["tiled", "plain"]


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_droplet48_100_steps(droplet48, path, store):
    wl, P, ref, bars = droplet48
    _check(_run(wl, 100, storage=store, path=path), P, ref, bars[store], f"droplet48 path={path}", store=store)


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_ragged_walled_bubble_ratio1000(path, store):
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    wl.noise, wl.seed = 0.005, 99
    P, ref = _oracle(wl, 60)
    _check(_run(wl, 60, storage=store, path=path), P, ref, _bars(wl, 60, store, P, ref),
           f"ragged walled bubble path={path}", store=store)


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_ragged_periodic_droplet_across_boundary(path, store):
    wl = inputs.static_droplet(L=24, radius=6.0, noise=0.01, seed=5)
    wl.nx, wl.ny, wl.nz = 45, 29, 27
    wl.center = (2.0, 27.5, 25.0)
    P, ref = _oracle(wl, 80)
    _check(_run(wl, 80, storage=store, path=path), P, ref, _bars(wl, 80, store, P, ref),
           f"ragged periodic droplet path={path}", store=store)


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_minimum_boxes(store):
    """4^3 periodic and 4 x 5 x 4 walled: every tile is ragged, every halo wraps, and a tile's
    lanes hold several copies of the same node (every node lies in the interface: 4 times the
    FP32 bars, plus the 16-bit stores' own derived term)."""
    for walled in (False, True):
        wl = inputs.static_droplet(L=4, radius=1.5, noise=0.01, seed=3)
        if walled:
            wl.ny, wl.wall_z, wl.gravity = 5, 1, (0.0, 0.0, -1e-5)
        P, ref = _oracle(wl, 10)
        bars = _bars(wl, 10, store, P, ref, factor=4.0)
        for path in PATHS:
            _check(_run(wl, 10, storage=store, path=path), P, ref, bars, f"minimum box walled={walled} path={path}",
                   store=store)


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_tiled_and_plain_kernels_agree(store):
    """FP32 moments, measured after 20 steps: max|d phi| ~ 2e-7, relative du and dp ~ 5e-7 (a halo
    or bounce-back error would show at 1e-3 or more).  16-bit moments: a last-bit difference of
    the collision can move a stored value across a 16-bit rounding boundary, so the two kernels
    are two realisations of the rounding: they agree to the FP32 bound plus 2 x SPREAD eps16 of
    the case."""
    walled = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    walled.noise, walled.seed = 0.005, 99
    periodic = inputs.static_droplet(L=24, radius=6.0, noise=0.01, seed=5)
    periodic.nx, periodic.ny, periodic.nz = 45, 29, 27
    for wl in (walled, periodic):
        P, ref = _oracle(wl, 20)
        eps = _eps16(wl, 20, store, P, ref)
        bars = tuple(t + 2 * SPREAD * e for t, e in zip((2e-6, 5e-6, 5e-6), eps))
        a, b = _run(wl, 20, storage=store, path=0), _run(wl, 20, storage=store, path=1)
        dphi = np.abs(a[0] - b[0]).max()
        du = np.abs(a[1] - b[1]).max() / np.abs(b[1]).max()
        dp = np.abs(a[2] - b[2]).max() / np.abs(b[2]).max()
        print(f"tiled vs plain store={store}: {dphi:.2e} {du:.2e} {dp:.2e}")
        assert dphi <= bars[0] and du <= bars[1] and dp <= bars[2]


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_z_split_does_not_change_the_result(store):
    """Each z chunk stages the plane below and above it from the same moments its neighbour
    chunk reads, so any split gives identical bits (1 chunk, uneven chunks, one plane each); the
    boxes have an odd and an even node count (16-bit halo words at either parity)."""
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    wl.noise, wl.seed = 0.005, 99
    ref = _run(wl, 12, storage=store, split=1)
    for split in (2, 3, 7, 19):
        _same(ref, _run(wl, 12, storage=store, split=split))
    pwl = inputs.static_droplet(L=24, radius=6.0, noise=0.01, seed=5)
    pref = _run(pwl, 12, storage=store, split=1)
    for split in (5, 24):
        _same(pref, _run(pwl, 12, storage=store, split=split))


def test_agrees_with_the_fp32_population_form():
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=21)
    a, b = _run(wl, 200), _run(wl, 200, storage=solver.LBM_FP32)
    assert np.abs(a[0] - b[0]).max() <= 1e-6
    assert np.abs(a[1] - b[1]).max() <= 1e-4 * np.abs(b[1]).max()
    assert np.abs(a[2] - b[2]).max() <= 1e-4 * np.abs(b[2]).max()
    assert np.abs(a[3] - b[3]).max() <= 1e-5 * np.abs(b[3]).max()


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_pstar_sum_is_conserved_like_the_fp32_form(store):
    """sum_i g_i = p* for any (rounded) a and B, so no storage drifts sum p* more than FP32 does."""
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=7)
    with solver.Solver(storage=store, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        o0 = s.observables()
        s.step(200)
        o = s.observables()
        g, _, _ = s.get_state()
    gsum = float(g.astype(np.float64).sum())
    assert math.isclose(o["sum_pstar"], gsum, rel_tol=1e-6, abs_tol=1e-6 * np.abs(g).sum())
    o32 = _run(wl, 200, storage=solver.LBM_FP32)[4]
    drift_m = abs(o["sum_pstar"] - o0["sum_pstar"])
    drift32 = abs(o32["sum_pstar"] - o0["sum_pstar"])
    print(f"sum p* drift over 200 steps: store {store} {drift_m:.3e}, FP32 populations {drift32:.3e}")
    assert drift_m <= 4 * drift32 + 1e-9 * s.n


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_state_round_trip_and_resume(store):
    """get_state expands the moments to FP32 g; set_state projects g back.  The projection is
    exact in exact arithmetic for these populations, so with FP32 moments the round trip changes a
    population by FP32 rounding only; with 16-bit moments a re-rounded a or B can move by one unit,
    bounded like the 16-bit population round trip (2 u16 times the largest deviation
    |g_i - w_i p*|).  A resumed run follows the uninterrupted one."""
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=11)
    with solver.Solver(storage=store, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(10)
        state = s.get_state()
        s.set_state(*state, step=10)
        again = s.get_state()
        s.step(15)
        a = s.read_fields()
        s.set_state(*state, step=10)
        s.step(15)
        b = s.read_fields()
        assert s.step_count == 25
    change = np.abs(again[0] - state[0]).max()
    if store == MOM:
        bound = 1e-6 * np.abs(state[0]).max()
    else:
        w1 = np.array([1 / 6, 2 / 3, 1 / 6])
        w = np.einsum("a,b,c->abc", w1, w1, w1).reshape(27, 1, 1, 1)
        g = state[0].astype(np.float64)
        dev = np.abs(g - w * g.sum(axis=0, keepdims=True)).max()
        bound = 2 * (2.0 ** -8 if store == solver.LBM_MOM_BF16 else 2.0 ** -11) * dev
    print(f"round trip store={store}: max population change {change:.3e} (bound {bound:.3e})")
    assert change <= bound
    assert np.array_equal(again[1], state[1]) and np.array_equal(again[2], state[2])
    assert np.abs(a[0] - b[0]).max() <= (1e-7 if store == MOM else 1e-6)
    assert np.abs(a[1] - b[1]).max() <= (1e-5 if store == MOM else 1e-3) * np.abs(a[1]).max()


def test_fp32_state_imported_into_moment_storage_continues_the_fp32_run():
    """A post-collision state of the FP32 population form lies in the span the moments describe,
    so importing it and stepping on tracks the FP32 run to FP32 rounding."""
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    wl.noise, wl.seed = 0.005, 99
    with solver.Solver(storage=solver.LBM_FP32, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(20)
        state = s.get_state()
        s.step(30)
        ref = s.read_fields()
    with solver.Solver(storage=MOM, **wl.params()) as s:
        s.set_state(*state, step=20)
        s.step(30)
        got = s.read_fields()
    assert np.abs(got[0] - ref[0]).max() <= 1e-6
    assert np.abs(got[1] - ref[1]).max() <= 1e-4 * np.abs(ref[1]).max()
    assert np.abs(got[2] - ref[2]).max() <= 1e-4 * np.abs(ref[2]).max()


def test_device_pointer_state_matches_host():
    import torch
    wl = inputs.static_droplet(L=20, radius=5.0, noise=0.01, seed=2)
    with solver.Solver(storage=MOM, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(5)
        g_host, phi, u = s.get_state()
        g_dev = torch.empty(27 * s.n, device="cuda")
        phi_d = torch.from_numpy(phi).cuda().reshape(-1)
        u_d = torch.from_numpy(u).cuda().reshape(-1)
        assert solver.load().lbm_get_state(s._ctx, g_dev.data_ptr(), None, None, 1) == 0
        assert np.array_equal(g_dev.cpu().numpy(), g_host.reshape(-1))
        s.set_state(g_dev, phi_d, u_d, step=5)
        from_dev = s.get_state()[0]
        s.set_state(g_host, phi, u, step=5)
        from_host = s.get_state()[0]
    # one FP64 sum over 27 directions vs three partial sums rounded to FP32
    assert np.abs(from_dev - from_host).max() <= 1e-6 * np.abs(from_host).max()


def test_fused_path_rejects_moment_storage():
    wl = inputs.static_droplet(L=16, radius=4.0)
    with solver.Solver(storage=MOM, **wl.params()) as s:
        s.set_path(0)
        s.set_path(1)
        with pytest.raises(solver.LbmError) as e:
            s.set_path(2)
        assert e.value.status == -1


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_rising_bubble_full_size_two_steps(store):
    """The benchmark workload (128 x 128 x 256, ratios 1000 / 100) in the benchmark's launch
    configuration, two steps against the oracle."""
    wl = inputs.rising_bubble()
    P, ref = _oracle(wl, 2)
    # velocities are ~1e-6 after two steps: measured against the velocity scale sqrt(gR) = 0.04
    bars = _bars(wl, 2, store, P, ref, u_scale=0.04)
    _check(_run(wl, 2, storage=store), P, ref, bars, "bubble full size", store=store, u_scale=0.04)


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_long_run_small_rising_bubble_observables(store):
    wl = inputs.rising_bubble(nx=24, ny=24, nz=96, R=5.0, zc=14.0, Eo=10.0, Mo=1e-2, rho_ratio=100.0,
                              mu_ratio=10.0, sqrt_gR=0.04, mobility=0.1)
    P, ref = _oracle(wl, 800)
    o, obs = oracle.observables(P, ref), _run(wl, 800, storage=store)[4]
    rise_o = o["centroid_gas"][2] - 14.0
    rise_g = obs["centroid_gas"][2] - 14.0
    print(f"rise oracle {rise_o:.5f} gpu {rise_g:.5f}")
    assert abs(rise_g / rise_o - 1) < 5e-3
    assert abs(obs["vel_gas"][2] / o["vel_gas"][2] - 1) < 5e-3
    assert abs(obs["mass"] / o["mass"] - 1) < 5e-3
    assert abs(obs["sum_phi"] / o["sum_phi"] - 1) < 5e-3


@pytest.mark.parametrize("store", STORES, ids=STORE_IDS)
def test_laplace_law(store):
    """Static droplet, 48^3, R = 12: p_in - p_out -> 2 sigma / R_eff, equal to the FP32 population
    form's to 1e-4 (FP32 moments) or 1e-3 (16-bit moments, the 16-bit population bar)."""
    wl = inputs.static_droplet(L=48, radius=12.0)
    ratios = {}
    for st in (solver.LBM_FP32, store):
        with solver.Solver(storage=st, **wl.params()) as s:
            s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
            s.step(4000)
            o = s.observables()
        reff = (3 * o["sum_phi"] / (4 * math.pi)) ** (1 / 3)
        ratios[st] = (o["p_liq"] - o["p_gas"]) / (2 * wl.sigma / reff)
    print(f"Laplace ratio FP32 {ratios[solver.LBM_FP32]:.5f} store={store} {ratios[store]:.5f}")
    assert abs(ratios[store] - 1) < 0.05
    assert abs(ratios[store] - ratios[solver.LBM_FP32]) < (1e-4 if store == MOM else 1e-3)
