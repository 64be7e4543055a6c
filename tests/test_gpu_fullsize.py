"""Parity at the full benchmark sizes, on sampled nodes.

The FP64 oracle cannot step a whole 512^3 box, but one step of a node depends only on the state
within three nodes of it: pull streaming reads g at distance 1, the forces use phi^{n+1} at
distance 1, and the Allen–Cahn update builds phi^{n+1} from phi^n and ubar^n at distance 2 (its
flux is a stencil of those).  So the GPU state after k steps of the full box is read out on the
device, a 7^3 neighbourhood of each sampled node is stepped once by the oracle (periodic on the
7^3 box; only the centre is used, and nothing it depends on wraps), and the centre's phi, u and p
are compared with the GPU's step k+1 of the full box, in the benchmark's launch configuration.
Nodes are drawn at random and from the interface (0.1 < phi < 0.9); on the walled bubble they
keep three planes from the walls.

One step from the same state differs only by FP32 rounding, for every storage (the 16-bit and
moment formats hand the oracle the populations they encode, and p* is carried exactly), so every
storage is held to the same bars: |d phi| <= 1e-6, |d u| <= 1e-4 max|u|, |d p| <= 1e-5 max|p|.
The velocity bar is the 100-step parity bar: on the droplet at rest max|u| is only the spurious
current, and the moment kernels' separable phi stencils (not in difference form) carry a larger
FP32 error into the surface force.  Measured on B300: populations |du|/max|u| <= 4e-6, moments
<= 2.2e-5; phi <= 5e-8 and p <= 3e-7 everywhere.
"""
import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu

SAMPLES = 48


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    solver.load()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _sample_nodes(phi, rng, zmargin):
    nz, ny, nx = phi.shape
    inter = np.argwhere((phi > 0.1) & (phi < 0.9))
    inter = inter[(inter[:, 0] >= zmargin) & (inter[:, 0] < nz - zmargin)]
    pick = inter[rng.choice(len(inter), SAMPLES // 2, replace=False)]
    rnd = np.stack([rng.integers(zmargin, nz - zmargin, SAMPLES // 2), rng.integers(0, ny, SAMPLES // 2),
                    rng.integers(0, nx, SAMPLES // 2)], axis=1)
    return np.concatenate([pick, rnd])


def _check_sampled(wl, store, k, zmargin):
    import torch
    N = wl.nx * wl.ny * wl.nz
    shape = (wl.nz, wl.ny, wl.nx)
    ps0 = wl.pstar_init()
    with solver.Solver(storage=store, **wl.params()) as s:
        s.init_fields(_f32(wl.phi0()), _f32(wl.u0()), None if ps0 is None else _f32(ps0))
        s.step(k)
        g = torch.empty(27 * N, device="cuda")
        phi_k = torch.empty(N, device="cuda")
        u_k = torch.empty(3 * N, device="cuda")
        assert solver.load().lbm_get_state(s._ctx, g.data_ptr(), phi_k.data_ptr(), u_k.data_ptr(), 1) == 0
        s.step(1)
        phi1 = torch.empty(N, device="cuda")
        u1 = torch.empty(3 * N, device="cuda")
        p1 = torch.empty(N, device="cuda")
        s.read_fields(phi1, u1, p1)
        torch.cuda.synchronize()
    g, phi_k, u_k = g.view(27, *shape), phi_k.view(*shape), u_k.view(3, *shape)
    phi1, u1, p1 = phi1.view(*shape), u1.view(3, *shape), p1.view(*shape)
    umax = float(u1.abs().max())
    pmax = float(p1.abs().max())
    prm = wl.params()
    P7 = oracle.Params(7, 7, 7, wall_z=0, **{q: v for q, v in prm.items()
                                             if q not in ("nx", "ny", "nz", "wall_z", "storage")})
    rng = np.random.default_rng(2501)
    nodes = _sample_nodes(phi_k.cpu().numpy(), rng, zmargin)
    worst = np.zeros(3)
    for z, y, x in nodes:
        zz = torch.tensor([(z + d) % wl.nz for d in range(-3, 4)], device="cuda")
        yy = torch.tensor([(y + d) % wl.ny for d in range(-3, 4)], device="cuda")
        xx = torch.tensor([(x + d) % wl.nx for d in range(-3, 4)], device="cuda")
        ix = (zz[:, None, None], yy[None, :, None], xx[None, None, :])
        sub = oracle.State(g[(slice(None),) + ix].double().cpu().numpy(), phi_k[ix].double().cpu().numpy(),
                           u_k[(slice(None),) + ix].double().cpu().numpy())
        out = oracle.step(P7, sub)
        ref_p = oracle.pressure(P7, out)[3, 3, 3]
        dphi = abs(float(phi1[z, y, x]) - out.phi[3, 3, 3])
        du = float(np.abs(u1[:, z, y, x].double().cpu().numpy() - out.u[:, 3, 3, 3]).max())
        dp = abs(float(p1[z, y, x]) - ref_p)
        worst = np.maximum(worst, [dphi, du / umax, dp / pmax])
    print(f"{wl.name} store={store} step {k}+1, {len(nodes)} nodes: max|dphi| {worst[0]:.2e}, "
          f"|du|/max|u| {worst[1]:.2e}, |dp|/max|p| {worst[2]:.2e}")
    assert worst[0] <= 1e-6 and worst[1] <= 1e-4 and worst[2] <= 1e-5


@pytest.fixture(scope="module")
def droplet512():
    return inputs.static_droplet(L=512)


@pytest.mark.parametrize("store", [solver.LBM_FP32, solver.LBM_BF16, solver.LBM_FP16, solver.LBM_MOM,
                                   solver.LBM_MOM_BF16, solver.LBM_MOM_FP16],
                         ids=["fp32", "bf16", "fp16", "mom", "mom_bf16", "mom_fp16"])
def test_droplet_512_sampled_step(droplet512, store):
    """The 512^3 static droplet of the sweep and of the precision study, 20 steps in."""
    _check_sampled(droplet512, store, 20, 0)


@pytest.mark.parametrize("store", [solver.LBM_FP32, solver.LBM_BF16, solver.LBM_MOM_BF16],
                         ids=["fp32", "bf16", "mom_bf16"])
def test_rising_bubble_sampled_step(store):
    """The 128 x 128 x 256 benchmark bubble (walls on z, ratios 1000 / 100), 60 steps in, when the
    flow has developed from rest."""
    _check_sampled(inputs.rising_bubble(), store, 60, 3)
