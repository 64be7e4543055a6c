"""lbm_observables_noalloc: the diagnostics entry point for callers that cannot allocate device
memory (an application that owns the whole device heap, or code that must not trigger the device
synchronisation a cudaMalloc implies).  It must give the same diagnostics as lbm_observables on
the same state, call after call, using only the library's built-in scratch array.

This file is collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu

FIELDS = ["sum_phi", "mass", "sum_pstar", "momentum", "centroid_liq", "centroid_gas", "vel_liq", "vel_gas",
          "p_liq", "p_gas", "n_liq", "n_gas", "umax", "phi_min", "phi_max", "n_nonfinite"]


def _close(a, b):
    a, b = np.atleast_1d(a), np.atleast_1d(b)
    return all(math.isclose(x, y, rel_tol=1e-12, abs_tol=1e-15) for x, y in zip(a, b))


def test_noalloc_observables_match_context_observables():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    L = solver.load()
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=21)
    wl.nx = 40                                   # not a multiple of the tile width
    s = solver.from_workload(wl)
    try:
        s.step(30)
        ref = s.observables()
        n = s.n
        g = torch.empty(27 * n, device="cuda")
        phi = torch.empty(n, device="cuda")
        u = torch.empty(3 * n, device="cuda")
        assert L.lbm_get_state(s._ctx, g.data_ptr(), phi.data_ptr(), u.data_ptr(), 1) == 0
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = solver.LbmObs()
            st = L.lbm_observables_noalloc(g.data_ptr(), phi.data_ptr(), u.data_ptr(), wl.nx, wl.ny, wl.nz,
                                           wl.rho_l, wl.rho_g, stream, ctypes.byref(out))
            assert st == 0, L.lbm_last_error()
            got = out.as_dict()
            for f in FIELDS:
                assert _close(got[f], ref[f]), (call, f, got[f], ref[f])
            assert got["step"] == 0.0
        # a box beyond the maximum size is rejected before any device work
        out = solver.LbmObs()
        st = L.lbm_observables_noalloc(g.data_ptr(), phi.data_ptr(), u.data_ptr(), 2048, 2048, 512,
                                       wl.rho_l, wl.rho_g, stream, ctypes.byref(out))
        assert st == -1 and b"maximum" in L.lbm_last_error()
    finally:
        s.close()
