"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs.  Both sides start from identical FP32 bytes (phi0, u0 rounded to float32, then widened
to FP64 for the oracle).

Tolerances (after the stated number of steps, FP32 on the GPU):
  max |d phi| <= 1e-5;  ||d u||_inf / ||u_oracle||_inf <= 1e-4;  ||d p||_inf / ||p_oracle||_inf <= 1e-4
and integral observables within 0.5% on long runs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu

TOL_PHI, TOL_U, TOL_P = 1e-5, 1e-4, 1e-4


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


def _gpu_run(wl, nsteps, path=0, chunk=0, phi0=None, u0=None):
    phi0 = wl.phi0() if phi0 is None else phi0
    u0 = wl.u0() if u0 is None else u0
    with solver.Solver(**wl.params()) as s:
        s.set_path(path)
        s.set_split(chunk)
        s.init_fields(_f32(phi0), _f32(u0), _pstar0(wl))
        s.step(nsteps)
        phi, u, p = s.read_fields()
        g, _, _ = s.get_state()
        obs = s.observables()
    return phi, u, p, g, obs


def _oracle_run(wl, nsteps, phi0=None, u0=None):
    phi0 = wl.phi0() if phi0 is None else phi0
    u0 = wl.u0() if u0 is None else u0
    P = oracle.Params(**wl.params())
    ps = _pstar0(wl)
    s = oracle.run(P, oracle.init(P, _f32(phi0).astype(np.float64), _f32(u0).astype(np.float64),
                                  None if ps is None else ps.astype(np.float64)), nsteps)
    return P, s


def _compare(gpu, P, ref):
    phi, u, p = gpu[:3]
    pref = oracle.pressure(P, ref)
    dphi = float(np.abs(phi - ref.phi).max())
    du = float(np.abs(u - ref.u).max() / np.abs(ref.u).max())
    dp = float(np.abs(p - pref).max() / np.abs(pref).max())
    return dphi, du, dp


def _assert_parity(gpu, P, ref, label):
    dphi, du, dp = _compare(gpu, P, ref)
    print(f"{label}: max|dphi| {dphi:.3e}  rel du {du:.3e}  rel dp {dp:.3e}")
    assert dphi <= TOL_PHI, (label, dphi)
    assert du <= TOL_U, (label, du)
    assert dp <= TOL_P, (label, dp)


# -- the 48^3 static droplet (density ratio 10, viscosity ratio 10), seeded velocity noise ---------

@pytest.fixture(scope="module")
def droplet48():
    wl = inputs.static_droplet(L=48, radius=12.0, noise=0.01, seed=1234)
    P, ref = _oracle_run(wl, 100)
    return wl, P, ref


PATHS = [0, 1, 2]
PATH_IDS = ["two_kernel", "three_kernel", "fused"]


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_droplet48_100_steps(droplet48, path):
    wl, P, ref = droplet48
    gpu = _gpu_run(wl, 100, path=path)
    _assert_parity(gpu, P, ref, f"droplet48 path={path}")
    # populations too (same velocity ordering on both sides)
    assert np.abs(gpu[3] - ref.g).max() <= 1e-4 * np.abs(ref.g).max()


def test_droplet48_observables(droplet48):
    wl, P, ref = droplet48
    phi, u, p, g, obs = _gpu_run(wl, 100)
    o = oracle.observables(P, ref)
    assert abs(obs["sum_phi"] / o["sum_phi"] - 1) < 1e-6
    assert abs(obs["mass"] / o["mass"] - 1) < 1e-6
    for a in range(3):
        assert abs(obs["centroid_liq"][a] - o["centroid_liq"][a]) < 1e-4
    assert abs(obs["umax"] / o["umax"] - 1) < 1e-4
    # the device reduction equals FP64 sums of the device's own fields
    phi64 = phi.astype(np.float64)
    rho = P.rho_l * phi64 + (1 - phi64) * P.rho_g
    assert math.isclose(obs["sum_phi"], phi64.sum(), rel_tol=1e-12)
    assert math.isclose(obs["mass"], rho.sum(), rel_tol=1e-12)
    assert math.isclose(obs["sum_pstar"], g.astype(np.float64).sum(), rel_tol=1e-9, abs_tol=1e-9)
    for a in range(3):
        assert math.isclose(obs["momentum"][a], (rho * u[a]).sum(), rel_tol=1e-9, abs_tol=1e-12)


@pytest.fixture(scope="module")
def droplet48_rest():
    wl = inputs.static_droplet(L=48, radius=12.0)
    P, ref100 = _oracle_run(wl, 100)
    ref200 = oracle.run(P, ref100, 100)
    return wl, P, ref100, ref200


@pytest.mark.parametrize("path", [0, 2], ids=["two_kernel", "fused"])
def test_droplet48_at_rest(droplet48_rest, path):
    """The configuration as stated (fluid at rest, checked after 100 and after 200 steps): only
    spurious currents move (max|u| ~ 9e-5), so the velocity tolerance is the strictest here.
    Before the sharpening weight was read as max(phi(1-phi), 0) (reading R15) an overshoot of phi
    above 1 at the droplet centre, where the normal is undefined, made FP32 and FP64 differ by
    1e-4 in phi."""
    wl, P, ref100, ref200 = droplet48_rest
    with solver.Solver(**wl.params()) as s:
        s.set_path(path)
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(100)
        gpu100 = s.read_fields()
        s.step(100)
        gpu200 = s.read_fields()
    _assert_parity(gpu100, P, ref100, f"droplet48 at rest, 100 steps, path={path}")
    dphi, du, dp = _compare(gpu200, P, ref200)
    print(f"droplet48 at rest, 200 steps, path={path}: max|dphi| {dphi:.3e} rel du {du:.3e} rel dp {dp:.3e} "
          f"(umax {np.abs(ref200.u).max():.2e})")
    assert dphi <= TOL_PHI and dp <= TOL_P
    assert du <= TOL_U


# -- ragged sizes, walls, density ratio 1000 --------------------------------------------------

def _ragged_bubble():
    wl = inputs.rising_bubble(nx=37, ny=21, nz=19, R=5.0, zc=8.0, sqrt_gR=0.04, mobility=0.1)
    wl.noise, wl.seed = 0.005, 99
    return wl


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_ragged_walled_bubble_ratio1000(path):
    wl = _ragged_bubble()
    P, ref = _oracle_run(wl, 60)
    gpu = _gpu_run(wl, 60, path=path)
    _assert_parity(gpu, P, ref, f"ragged walled bubble path={path}")


@pytest.mark.parametrize("path", [0, 2], ids=["two_kernel", "fused"])
def test_ragged_periodic_droplet_across_boundary(path):
    wl = inputs.static_droplet(L=24, radius=6.0, noise=0.01, seed=5)
    wl.nx, wl.ny, wl.nz = 45, 29, 27
    wl.center = (2.0, 27.5, 25.0)            # wraps around all three periodic boundaries
    P, ref = _oracle_run(wl, 80)
    gpu = _gpu_run(wl, 80, path=path)
    _assert_parity(gpu, P, ref, f"ragged periodic droplet path={path}")


@pytest.mark.parametrize("path", [0, 2], ids=["two_kernel", "fused"])
def test_minimum_box(path):
    wl = inputs.static_droplet(L=4, radius=1.5, noise=0.01, seed=3)
    P, ref = _oracle_run(wl, 10)
    _assert_parity(_gpu_run(wl, 10, path=path), P, ref, "4^3 box")
    wl = inputs.static_droplet(L=4, radius=1.5, noise=0.01, seed=3)
    wl.ny, wl.wall_z, wl.gravity = 5, 1, (0.0, 0.0, -1e-5)
    P, ref = _oracle_run(wl, 10)
    _assert_parity(_gpu_run(wl, 10, path=path), P, ref, "4x5x4 walled box")


# -- boxes whose x extent is a multiple of 128 take the vector Allen–Cahn kernel ---------------

def _wide_box(which):
    if which == "128_walled":
        # the warp spans the whole periodic row: the x halo is the shuffle wrap-around
        wl = inputs.rising_bubble(nx=128, ny=11, nz=20, R=3.5, zc=8.0, sqrt_gR=0.04, mobility=0.1)
        wl.center = (126.5, 5.0, 8.0)            # across the periodic x boundary
        wl.noise, wl.seed = 0.005, 41
    else:
        # two warps per row: lanes 0 and 31 load the halo columns; odd ny leaves a ragged row tile
        wl = inputs.rising_bubble(nx=256, ny=5, nz=12, R=3.0, zc=6.0, sqrt_gR=0.04, mobility=0.1,
                                  rho_ratio=100.0)
        wl.wall_z = 0
        wl.center = (128.0, 2.0, 11.0)           # across the tile boundary x = 128 and the periodic z
        wl.noise, wl.seed = 0.005, 42
    return wl


@pytest.mark.parametrize("which", ["128_walled", "256_periodic"])
def test_wide_boxes_vector_allen_cahn(which):
    wl = _wide_box(which)
    P, ref = _oracle_run(wl, 40)
    _assert_parity(_gpu_run(wl, 40), P, ref, f"{which} box")
    a = _gpu_run(wl, 13, chunk=0)
    for chunk in (1, 5):
        b = _gpu_run(wl, 13, chunk=chunk)
        for x, y in zip(a[:4], b[:4]):
            assert np.array_equal(x, y), chunk


# -- determinism and invariances of the fused kernel -------------------------------------------

@pytest.mark.parametrize("path", [0, 2], ids=["two_kernel", "fused"])
def test_work_split_does_not_change_results(path):
    """The number of z chunks per column tile changes only how the planes are split among
    CTAs; halo planes are recomputed with identical arithmetic, so results are bit-identical."""
    wl = _ragged_bubble()
    ref = _gpu_run(wl, 25, path=path, chunk=0)
    for chunk in (1, 3, 7, 64):
        out = _gpu_run(wl, 25, path=path, chunk=chunk)
        for a, b in zip(ref[:4], out[:4]):
            assert np.array_equal(a, b), chunk


def test_checkpoint_resume_bit_exact():
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=11)
    with solver.Solver(**wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(10)
        state = s.get_state()
        s.step(15)
        a = s.get_state()
        s.set_state(*state, step=10)
        assert s.step_count == 10
        s.step(15)
        b = s.get_state()
        assert s.step_count == 25
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_device_pointers_match_host_pointers():
    import torch
    wl = inputs.static_droplet(L=20, radius=5.0, noise=0.01, seed=2)
    phi0, u0 = _f32(wl.phi0()), _f32(wl.u0())
    host = _gpu_run(wl, 5)
    ps = torch.from_numpy(_pstar0(wl)).cuda().reshape(-1)
    with solver.Solver(**wl.params()) as s:
        s.init_fields(torch.from_numpy(phi0).cuda().reshape(-1), torch.from_numpy(u0).cuda().reshape(-1), ps)
        s.step(5)
        out = [torch.empty(n, device="cuda") for n in (s.n, 3 * s.n, s.n)]
        s.read_fields(*out)
        torch.cuda.synchronize()
    for a, b in zip(host[:3], out):
        assert np.array_equal(a.reshape(-1), b.cpu().numpy())


@pytest.mark.parametrize("kind", ["default", "created"])
def test_kernels_run_on_the_callers_stream(kind):
    """Every kernel is enqueued on the stream given at creation (NULL = the legacy default stream):
    CUDA events recorded on that stream around the steps span their whole device time."""
    import time
    import torch
    st = torch.cuda.default_stream() if kind == "default" else torch.cuda.Stream()
    wl = inputs.static_droplet(L=128, radius=32.0)
    with torch.cuda.stream(st):
        s = solver.Solver(stream=st, **wl.params())
        try:
            s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
            s.step(5)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(st)
            s.step(60)
            e1.record(st)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            ev = e0.elapsed_time(e1) * 1e-3
        finally:
            s.close()
    print(f"stream {kind}: event {ev * 1e3:.2f} ms, wall {wall * 1e3:.2f} ms")
    assert ev > 0.7 * wall


# -- error paths ----------------------------------------------------------------------------------

def test_step_before_init_and_nonfinite_detection():
    wl = inputs.static_droplet(L=16, radius=4.0)
    with solver.Solver(**wl.params()) as s:
        with pytest.raises(solver.LbmError) as e:
            s.step(1)
        assert e.value.status == -6
        phi0 = _f32(wl.phi0())
        phi0[3, 4, 5] = np.nan
        s.init_fields(phi0, _f32(wl.u0()))
        s.step(2)
        with pytest.raises(solver.LbmError) as e:
            s.observables()
        assert e.value.status == -4
        o = s.observables(allow_nonfinite=True)
        assert o["n_nonfinite"] > 0


# -- the benchmark workload at full size, in the benchmark's launch configuration --------------

# 20 steps: the start-up flow is developed (max|u| ~ 0.1 in the gas) and the velocity is compared
# with the same relative bar as everywhere else.  Beyond ~25 steps this transient at density ratio
# 1000 amplifies rounding: the FP64 oracle started from inputs perturbed by one FP32 rounding
# (2^-24 relative) differs from itself by 5e-8 in phi after 20 steps but 4e-6 after 30 and 5e-5
# after 40, so no FP32 result can be held to 1e-5 there.
FULL_STEPS = 20


@pytest.fixture(scope="module")
def bubble_full():
    wl = inputs.rising_bubble()          # 128 x 128 x 256, walls on z, ratios 1000 / 100
    P, ref = _oracle_run(wl, FULL_STEPS)
    return wl, P, ref


@pytest.mark.parametrize("path", [0, 2], ids=["two_kernel", "fused"])
def test_rising_bubble_full_size(bubble_full, path):
    """The whole benchmark box, element by element against the oracle after 20 steps, in the
    benchmark's launch configuration (path 0) and with the fused kernel (path 2), at the FP32 bars
    (phi absolute, u and p relative to their maxima)."""
    wl, P, ref = bubble_full
    gpu = _gpu_run(wl, FULL_STEPS, path=path)
    assert np.abs(ref.u).max() > 1e-4
    _assert_parity(gpu, P, ref, f"rising bubble 128x128x256, {FULL_STEPS} steps, path {path}")


# -- long runs: integral observables within 0.5% ---------------------------------------------------

def test_long_run_small_rising_bubble_observables():
    wl = inputs.rising_bubble(nx=24, ny=24, nz=96, R=5.0, zc=14.0, Eo=10.0, Mo=1e-2, rho_ratio=100.0,
                              mu_ratio=10.0, sqrt_gR=0.04, mobility=0.1)
    nsteps = 800
    P, ref = _oracle_run(wl, nsteps)
    gpu = _gpu_run(wl, nsteps)
    o, obs = oracle.observables(P, ref), gpu[4]
    rise_o = o["centroid_gas"][2] - 14.0
    rise_g = obs["centroid_gas"][2] - 14.0
    print(f"bubble rise oracle {rise_o:.5f} gpu {rise_g:.5f}; vel {o['vel_gas'][2]:.3e} {obs['vel_gas'][2]:.3e}")
    assert rise_o > 0.1
    assert abs(rise_g / rise_o - 1) < 5e-3
    assert abs(obs["vel_gas"][2] / o["vel_gas"][2] - 1) < 5e-3
    assert abs(obs["mass"] / o["mass"] - 1) < 5e-3
    assert abs(obs["sum_phi"] / o["sum_phi"] - 1) < 5e-3


def test_laplace_law_on_gpu():
    """Static droplet, 48^3, R = 12: p_in - p_out -> 2 sigma / R_eff (closed form)."""
    wl = inputs.static_droplet(L=48, radius=12.0)
    with solver.Solver(**wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl))
        s.step(4000)
        o = s.observables()
    reff = (3 * o["sum_phi"] / (4 * math.pi)) ** (1 / 3)
    ratio = (o["p_liq"] - o["p_gas"]) / (2 * wl.sigma / reff)
    print(f"Laplace 48^3 R=12: dp ratio {ratio:.4f}, umax {o['umax']:.2e}")
    assert abs(ratio - 1) < 0.05


def test_literal_advection_form_on_path_1():
    """lbm_set_advection(ctx, 1): the paper's literal ubar . G[phi] advection on the unfused path,
    against the oracle with the same form (advect = 1), 100 steps on the noise droplet, whose
    velocity field is not divergence-free.  Sum phi is no longer an invariant: the GPU's drift
    follows the oracle's.  The form is refused on paths 0 and 2."""
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.02, seed=17)
    phi0, u0, ps = _f32(wl.phi0()), _f32(wl.u0()), _pstar0(wl)
    P = oracle.Params(**wl.params())
    P.advect = 1
    ref = oracle.run(P, oracle.init(P, phi0.astype(np.float64), u0.astype(np.float64),
                                    None if ps is None else ps.astype(np.float64)), 100)
    with solver.Solver(**wl.params()) as s:
        with pytest.raises(solver.LbmError):
            s.set_advection(1)            # path 0
        s.set_path(1)
        s.set_advection(1)
        for path in (0, 2):
            with pytest.raises(solver.LbmError):
                s.set_path(path)
        s.init_fields(phi0, u0, ps)
        s.step(100)
        phi, u, p = s.read_fields()
    _assert_parity((phi, u, p), P, ref, "literal advection path 1")
    drift_o = ref.phi.sum() - phi0.astype(np.float64).sum()
    drift_g = phi.astype(np.float64).sum() - phi0.astype(np.float64).sum()
    print(f"sum phi drift over 100 steps: oracle {drift_o:.6e}, GPU {drift_g:.6e}")
    assert abs(drift_o) > 1e-4
    assert abs(drift_g - drift_o) <= 1e-3 * abs(drift_o) + 1e-4
