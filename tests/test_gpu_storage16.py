"""16-bit population storage (LBM_BF16, LBM_FP16) against the FP64 oracle and the FP32 path.

The 16-bit formats round only h_i = (g_i - f^eq_i(p*, u)) / w_i, the non-equilibrium part of each
population, once per step; p*, u and phi stay FP32 and the arithmetic is FP32.  The oracle
emulates exactly that rounding (oracle.Params.storage16, pinned against the format's definition
in test_oracle_storage16.py).  So each case's bar is derived, not fitted: the format's own effect
on it, eps16 = |oracle with 16-bit storage - oracle| (max|d phi|, relative du, relative dp), is
computed by the oracle at test time, and a GPU run must lie within

    FP32 bar (1e-5 / 1e-4 / 1e-4, the FP32 path's bars)  +  3 eps16

of the plain oracle.  The factor: a GPU run is another realisation of the same rounding (a
last-bit difference in FP32 moves a value across a rounding boundary, and the runs' rounding
errors decorrelate from there), so its distance from the plain oracle is of the size of eps16,
not below it; measured on B300 within 1.5 eps16 on every case here (droplet 48^3 100 steps,
ragged walled bubble at density ratio 1000 60 steps, ragged periodic droplet 80 steps; BF16 and
FP16, both kernels).  Integral observables (rise, bubble velocity, mass, sum phi) stay within the
0.5% bar of the FP32 form on long runs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu

STORAGES = [solver.LBM_BF16, solver.LBM_FP16]
IDS = ["bf16", "fp16"]
FP32_BAR = (1e-5, 1e-4, 1e-4)   # the FP32 path's bars against the oracle: max|d phi|, rel du, rel dp
SPREAD = 3.0                    # an independent realisation of the rounding: measured within 1.5 eps16


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


def _run(wl, nsteps, storage, path=0):
    with solver.Solver(storage=storage, **wl.params()) as s:
        s.set_path(path)
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


def _reference(wl, nsteps, storage, u_scale=None):
    """(P, ref, bars): the plain oracle run and the derived bars FP32 bar + SPREAD eps16, eps16
    the emulated 16-bit oracle's distance from it."""
    P, ref = _oracle(wl, nsteps)
    P16, ref16 = _oracle(wl, nsteps, storage)
    eps = _errs((ref16.phi, ref16.u, oracle.pressure(P16, ref16)), P, ref, u_scale)
    return P, ref, tuple(FP32_BAR[j] + SPREAD * eps[j] for j in range(3))


def _check(out, P, ref, bars, label, u_scale=None):
    d = _errs(out, P, ref, u_scale)
    print(f"{label}: max|dphi| {d[0]:.3e} rel du {d[1]:.3e} rel dp {d[2]:.3e}; bars {bars[0]:.3e} {bars[1]:.3e} "
          f"{bars[2]:.3e}")
    assert all(d[j] <= bars[j] for j in range(3)), (label, d, bars)


@pytest.fixture(scope="module")
def droplet48():
    wl = inputs.static_droplet(L=48, radius=12.0, noise=0.01, seed=1234)
    return {st: (wl,) + _reference(wl, 100, st) for st in STORAGES}


# path 0: tiled 16-bit kernel (shared-memory staging); path 1: the plain one-node-per-thread kernel
PATHS = [0, 1]
PATH_IDS = ["tiled", "plain"]


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_droplet48_100_steps(droplet48, storage, path):
    wl, P, ref, bars = droplet48[storage]
    _check(_run(wl, 100, storage, path), P, ref, bars, f"droplet48 storage={storage} path={path}")


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_ragged_walled_bubble_ratio1000(storage, path):
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    wl.noise, wl.seed = 0.005, 99
    P, ref, bars = _reference(wl, 60, storage)
    _check(_run(wl, 60, storage, path), P, ref, bars, f"ragged walled bubble storage={storage} path={path}")


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_ragged_periodic_droplet_across_boundary(storage, path):
    wl = inputs.static_droplet(L=24, radius=6.0, noise=0.01, seed=5)
    wl.nx, wl.ny, wl.nz = 45, 29, 27
    wl.center = (2.0, 27.5, 25.0)
    P, ref, bars = _reference(wl, 80, storage)
    _check(_run(wl, 80, storage, path), P, ref, bars, f"ragged periodic droplet storage={storage} path={path}")


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_minimum_boxes(storage):
    """4^3 periodic and 4 x 5 x 4 walled: every tile is ragged and every halo wraps.  Every node
    of these boxes lies inside the interface of the R = 1.5, W = 4 droplet, where the
    non-equilibrium part h is largest relative to u; the derived bars follow that."""
    for walled in (False, True):
        wl = inputs.static_droplet(L=4, radius=1.5, noise=0.01, seed=3)
        if walled:
            wl.ny, wl.wall_z, wl.gravity = 5, 1, (0.0, 0.0, -1e-5)
        P, ref, bars = _reference(wl, 10, storage)
        for path in PATHS:
            _check(_run(wl, 10, storage, path), P, ref, bars,
                   f"minimum box storage={storage} walled={walled} path={path}")


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_tiled_and_plain_kernels_agree(storage):
    """The tiled and the plain 16-bit kernels do the same arithmetic on the same values, but the
    compiler may order FP32 operations differently, and a last-bit difference can move a value
    across a 16-bit rounding boundary, after which the two runs carry independent rounding
    errors.  So they agree as two realisations of the rounding, each within its derived bar of the
    oracle: to twice that bar, not bit for bit."""
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    wl.noise, wl.seed = 0.005, 99
    a, b = _run(wl, 20, storage, 0), _run(wl, 20, storage, 1)
    _, ref, bars = _reference(wl, 20, storage)
    assert np.abs(a[0] - b[0]).max() <= 2 * bars[0]
    assert np.abs(a[1] - b[1]).max() <= 2 * bars[1] * np.abs(ref.u).max()


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_pstar_sum_is_the_sum_of_the_rebuilt_populations(storage):
    """lbm_observables' sum p* (P + sum w h per node) equals the FP64 sum of the FP32 populations
    lbm_get_state rebuilds, and the step conserves it as well as the FP32 form does."""
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=7)
    with solver.Solver(storage=storage, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        o0 = s.observables()
        s.step(200)
        o = s.observables()
        g, _, _ = s.get_state()
    gsum = float(g.astype(np.float64).sum())
    assert math.isclose(o["sum_pstar"], gsum, rel_tol=1e-6, abs_tol=1e-6 * np.abs(g).sum())
    _, _, _, _, o32 = _run(wl, 200, solver.LBM_FP32)
    drift16 = abs(o["sum_pstar"] - o0["sum_pstar"])
    drift32 = abs(o32["sum_pstar"] - o0["sum_pstar"])
    print(f"sum p* drift over 200 steps: 16-bit {drift16:.3e}, FP32 {drift32:.3e}")
    assert drift16 <= 4 * drift32 + 1e-9 * s.n


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_state_round_trip_and_resume(storage):
    """get_state expands to FP32 g; set_state compresses it again.  The round trip is not bit
    exact: P is recomputed as sum g, whose FP32 rounding can move an h across a 16-bit rounding
    boundary, so a population may change by one 16-bit unit of its deviation.  A resumed run
    follows the uninterrupted one to the same level."""
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=11)
    with solver.Solver(storage=storage, **wl.params()) as s:
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
    # one 16-bit unit (2 u16) of the largest deviation |g_i - w_i p*| bounds the change
    w1 = np.array([1 / 6, 2 / 3, 1 / 6])
    w = np.einsum("a,b,c->abc", w1, w1, w1).reshape(27, 1, 1, 1)   # index 9(cz+1) + 3(cy+1) + (cx+1)
    g = state[0].astype(np.float64)
    dev = np.abs(g - w * g.sum(axis=0, keepdims=True)).max()
    u16 = 2.0 ** -8 if storage == solver.LBM_BF16 else 2.0 ** -11
    print(f"round trip: max change {np.abs(again[0] - state[0]).max():.3e}, bound {2 * u16 * dev:.3e}")
    assert np.abs(again[0] - state[0]).max() <= 2 * u16 * dev
    assert np.array_equal(again[1], state[1]) and np.array_equal(again[2], state[2])
    assert np.abs(a[0] - b[0]).max() <= 1e-6
    assert np.abs(a[1] - b[1]).max() <= 1e-3 * np.abs(a[1]).max()


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_device_pointer_state_matches_host(storage):
    import torch
    wl = inputs.static_droplet(L=20, radius=5.0, noise=0.01, seed=2)
    with solver.Solver(storage=storage, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(5)
        g_host, phi, u = s.get_state()
        g_dev = torch.empty(27 * s.n, device="cuda")
        phi_d = torch.from_numpy(phi).cuda().reshape(-1)
        u_d = torch.from_numpy(u).cuda().reshape(-1)
        st = solver.load().lbm_get_state(s._ctx, g_dev.data_ptr(), None, None, 1)
        assert st == 0
        assert np.array_equal(g_dev.cpu().numpy(), g_host.reshape(-1))
        # compressing from device and from host gives the same state
        s.set_state(g_dev, phi_d, u_d, step=5)
        from_dev = s.get_state()[0]
        s.set_state(g_host, phi, u, step=5)
        from_host = s.get_state()[0]
    assert np.array_equal(from_dev, from_host)


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_fused_path_rejects_16_bit_storage(storage):
    wl = inputs.static_droplet(L=16, radius=4.0)
    with solver.Solver(storage=storage, **wl.params()) as s:
        s.set_path(0)
        s.set_path(1)
        with pytest.raises(solver.LbmError) as e:
            s.set_path(2)
        assert e.value.status == -1


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_rising_bubble_full_size_two_steps(storage):
    """The benchmark workload (128 x 128 x 256, ratios 1000 / 100) in the benchmark's launch
    configuration, two steps against the oracle."""
    wl = inputs.rising_bubble()
    # velocities are ~1e-6 after two steps: measured against the velocity scale sqrt(gR) = 0.04
    P, ref, bars = _reference(wl, 2, storage, u_scale=0.04)
    _check(_run(wl, 2, storage), P, ref, bars, f"bubble full size storage={storage}", u_scale=0.04)


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_long_run_small_rising_bubble_observables(storage):
    wl = inputs.rising_bubble(nx=24, ny=24, nz=96, R=5.0, zc=14.0, Eo=10.0, Mo=1e-2, rho_ratio=100.0,
                              mu_ratio=10.0, sqrt_gR=0.04, mobility=0.1)
    P, ref = _oracle(wl, 800)
    o, obs = oracle.observables(P, ref), _run(wl, 800, storage)[4]
    rise_o = o["centroid_gas"][2] - 14.0
    rise_g = obs["centroid_gas"][2] - 14.0
    print(f"storage={storage}: rise oracle {rise_o:.5f} gpu {rise_g:.5f}")
    assert abs(rise_g / rise_o - 1) < 5e-3
    assert abs(obs["vel_gas"][2] / o["vel_gas"][2] - 1) < 5e-3
    assert abs(obs["mass"] / o["mass"] - 1) < 5e-3
    assert abs(obs["sum_phi"] / o["sum_phi"] - 1) < 5e-3


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_laplace_law(storage):
    """Static droplet, 48^3, R = 12: p_in - p_out -> 2 sigma / R_eff, and the 16-bit value equals
    the FP32 one to 1e-3."""
    wl = inputs.static_droplet(L=48, radius=12.0)
    ratios = {}
    for st in (solver.LBM_FP32, storage):
        with solver.Solver(storage=st, **wl.params()) as s:
            s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
            s.step(4000)
            o = s.observables()
        reff = (3 * o["sum_phi"] / (4 * math.pi)) ** (1 / 3)
        ratios[st] = (o["p_liq"] - o["p_gas"]) / (2 * wl.sigma / reff)
    print(f"Laplace ratio FP32 {ratios[solver.LBM_FP32]:.5f} storage={storage} {ratios[storage]:.5f}")
    assert abs(ratios[storage] - 1) < 0.05
    assert abs(ratios[storage] - ratios[solver.LBM_FP32]) < 1e-3


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_conversion_moves_each_population_by_at_most_its_rounded_deviation(storage):
    """The 16-bit format rounds only the deviation h_i = (g_i - f^eq_i(p*, u)) / w_i (Eq. eqts for
    f^eq) and keeps P = p* - sum_j w_j h_j(rounded), so that the expanded populations still sum to
    p*.  Loading an FP32 state (lbm_set_state) and expanding it again (lbm_get_state) therefore
    moves population i by at most w_i u16 |h_i| (its own rounding) plus w_i u16 sum_j w_j |h_j|
    (its share of the P correction), with u16 the format's unit roundoff, plus the FP32 rounding
    of the conversion arithmetic.  Checked at every population of a developed state (a walled
    bubble at density ratio 1000 after 30 FP32 steps, where the deviations are largest)."""
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    with solver.Solver(storage=solver.LBM_FP32, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(30)
        g32, phi, u = s.get_state()
    with solver.Solver(storage=storage, **wl.params()) as s:
        s.set_state(g32, phi, u, step=30)
        g16, phi16, u16_ = s.get_state()
    assert np.array_equal(phi16, phi) and np.array_equal(u16_, u)
    g = g32.astype(np.float64)
    ps = g.sum(axis=0)
    w1 = np.array([1 / 6, 2 / 3, 1 / 6])
    w = np.einsum("a,b,c->abc", w1, w1, w1).reshape(27)             # index 9(cz+1) + 3(cy+1) + (cx+1)
    feq = np.empty_like(g)
    uu = u.astype(np.float64)
    for idx in np.ndindex(ps.shape):                                   # the oracle's equilibrium, node by node
        feq[(slice(None),) + idx] = oracle.equilibrium(ps[idx], uu[(slice(None),) + idx])
    h = (g - feq) / w[:, None, None, None]
    unit = 2.0 ** -8 if storage == solver.LBM_BF16 else 2.0 ** -11
    tiny = 0.0 if storage == solver.LBM_BF16 else 2.0 ** -25 / 4096    # FP16 holds 2^12 h; subnormal spacing
    share = (w[:, None, None, None] * (unit * np.abs(h) + tiny)).sum(axis=0)
    bound = (w[:, None, None, None] * (unit * np.abs(h) + tiny) + w[:, None, None, None] * share
             + 8 * 2.0 ** -24 * (np.abs(g) + w[:, None, None, None] * np.abs(ps)))
    err = np.abs(g16.astype(np.float64) - g)
    print(f"storage {storage}: largest |change| / bound {float((err / bound).max()):.3f}, largest |h| "
          f"{float(np.abs(h).max()):.3e}")
    assert (err <= bound).all()
    assert err.max() > 0.05 * bound.max()     # the rounding is seen, not hidden under the slack


@pytest.mark.parametrize("storage", STORAGES, ids=IDS)
def test_z_split_does_not_change_the_result(storage):
    """The marching 16-bit kernel gives the same bits for every z split of its column tiles: a
    node's arithmetic does not depend on which block stages or completes it (walled ragged box)."""
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    out = []
    for split in (1, 3, 19):
        with solver.Solver(storage=storage, **wl.params()) as s:
            s.set_split(split)
            s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
            s.step(12)
            out.append((s.get_state()[0], s.read_fields()))
    for g, f in out[1:]:
        assert np.array_equal(g, out[0][0])
        for a, b in zip(f, out[0][1]):
            assert np.array_equal(a, b)
