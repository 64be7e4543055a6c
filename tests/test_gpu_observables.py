"""The FP64 diagnostics at sizes where every thread of the reduction handles many nodes.

The reduction adds a thread's terms exactly in FP32 pairs (TwoSum / TwoProduct) and moves them
into FP64 every 16 nodes, so boxes of a few thousand nodes (one node per thread) never reach a
mid-loop flush.  These cases do: an 8.4M-node box (about 28 nodes per thread) and a 1-D box of
2^24 + 37 nodes along x (about 55 per thread), whose x coordinates above 2^24 take the split
product.  Every field of lbm_obs is compared with its definition evaluated in FP64 on the same
FP32 fields: the sums of phi, mass, p* and momentum, the centroids and velocities to 1e-12
relative, the phase pressures (FP32 products of p* and rho) to 1e-6, max |u| to 1e-6, the counts
and phi extremes exactly.  The inputs are seeded random fields (phi spread over both phases and
the interface), written straight into device memory and read through lbm_observables_noalloc.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2501_00846_b300 import solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    solver.load()


def _reference(g, phi, u, nx, ny, nz, rho_l, rho_g):
    """The diagnostics by their definitions, in FP64 (torch reductions on the device)."""
    import torch
    n = nx * ny * nz
    ph = phi.double()
    uu = u.view(3, n).double()
    ps = torch.zeros(n, dtype=torch.float64, device="cuda")
    for i in range(27):
        ps += g[i * n:(i + 1) * n].double()
    rho = rho_g + (rho_l - rho_g) * ph
    k = torch.arange(n, device="cuda", dtype=torch.int64)
    coords = [(k % nx).double(), ((k // nx) % ny).double(), (k // (nx * ny)).double()]
    sphi = float(ph.sum())
    sgas = float((1.0 - ph).sum())
    p = ps * rho / 3.0
    liq, gas = ph > 0.999, ph < 0.001
    return {
        "sum_phi": sphi, "mass": float(rho.sum()), "sum_pstar": float(ps.sum()),
        "momentum": [float((rho * uu[a]).sum()) for a in range(3)],
        "centroid_liq": [float((ph * coords[a]).sum()) / sphi for a in range(3)],
        "centroid_gas": [float(((1.0 - ph) * coords[a]).sum()) / sgas for a in range(3)],
        "vel_liq": [float((ph * uu[a]).sum()) / sphi for a in range(3)],
        "vel_gas": [float(((1.0 - ph) * uu[a]).sum()) / sgas for a in range(3)],
        "n_liq": float(liq.sum()), "n_gas": float(gas.sum()),
        "p_liq": float(p[liq].mean()), "p_gas": float(p[gas].mean()),
        "umax": float(torch.sqrt((uu * uu).sum(0)).max()),
        "phi_min": float(ph.min()), "phi_max": float(ph.max()),
    }


@pytest.mark.parametrize("shape", [(256, 256, 128), ((1 << 24) + 37, 1, 1)], ids=["8M_box", "x_beyond_2^24"])
def test_diagnostics_match_fp64_definitions_at_scale(shape):
    import torch
    nx, ny, nz = shape
    n = nx * ny * nz
    rho_l, rho_g = 1.0, 0.001
    gen = torch.Generator(device="cuda").manual_seed(2501)
    # phi: a third liquid (>= 0.9995), a third gas (<= 0.0005), a third interface, slight over/undershoot
    sel = torch.randint(0, 3, (n,), generator=gen, device="cuda")
    r = torch.rand(n, generator=gen, device="cuda")
    phi = torch.where(sel == 0, 0.9995 + 0.0010 * r, torch.where(sel == 1, -0.0005 + 0.0010 * r, r)).float()
    u = (0.02 * torch.randn(3 * n, generator=gen, device="cuda")).float()
    g = (0.01 * torch.randn(27 * n, generator=gen, device="cuda") + 1.0 / 27.0).float()
    ref = _reference(g, phi, u, nx, ny, nz, rho_l, rho_g)
    L = solver.load()
    out = solver.LbmObs()
    st = L.lbm_observables_noalloc(g.data_ptr(), phi.data_ptr(), u.data_ptr(), nx, ny, nz, rho_l, rho_g,
                                   torch.cuda.current_stream().cuda_stream, ctypes.byref(out))
    assert st == 0, L.lbm_last_error()
    got = out.as_dict()
    for f in ("sum_phi", "mass", "sum_pstar", "momentum", "centroid_liq", "centroid_gas", "vel_liq", "vel_gas"):
        for a, b in zip(np.atleast_1d(got[f]), np.atleast_1d(ref[f])):
            assert math.isclose(a, b, rel_tol=1e-12, abs_tol=1e-12 * n), (f, a, b)
    for f in ("p_liq", "p_gas", "umax"):
        assert math.isclose(got[f], ref[f], rel_tol=1e-6), (f, got[f], ref[f])
    for f in ("n_liq", "n_gas", "phi_min", "phi_max"):
        assert got[f] == ref[f], (f, got[f], ref[f])
    assert got["n_nonfinite"] == 0.0
