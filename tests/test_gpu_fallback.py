"""The fine solver as the fallback of the corrected coarse run.

lbm_prolong2_state: every field of the fine state equals its cell-centred trilinear definition
(3/4 of the parent cell and 1/4 of the neighbour the fine node lies towards, per axis), evaluated in
FP64 on the same coarse state, on ragged periodic and walled boxes; the fine sums of phi, p* and
ubar are 8 times the coarse ones.

closure.run_with_fallback: a network whose velocity correction is far too large trips the checks
of the corrected run; the run then continues from its last good checkpoint on the fine grid, and
its final state is the one of that checkpoint prolonged and advanced by the plain fine solver, bit
for bit.  A network that corrects nothing passes every check and never falls back.
"""
import numpy as np
import pytest

from paper_2501_00846_b300 import closure, inputs, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    solver.load()


def _prolong_reference(a, wall):
    """Cell-centred 2x prolongation of a [..., nz, ny, nx] array along its last three axes."""
    out = np.asarray(a, np.float64)
    for ax, clamp in ((-1, False), (-2, False), (-3, wall)):
        n = out.shape[ax]
        i = np.arange(2 * n) // 2
        j = np.where(np.arange(2 * n) % 2 == 1, i + 1, i - 1)
        j = np.clip(j, 0, n - 1) if clamp else j % n
        out = 0.75 * np.take(out, i, axis=ax) + 0.25 * np.take(out, j, axis=ax)
    return out


@pytest.mark.parametrize("shape,wall", [((10, 6, 5), 0), ((8, 4, 8), 1)], ids=["periodic_ragged", "walled"])
def test_prolongation_matches_its_definition(shape, wall):
    nx, ny, nz = shape
    rng = np.random.default_rng(11)
    common = dict(rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.01, width=4.0, mobility=0.1, wall_z=wall)
    with solver.Solver(nx=nx, ny=ny, nz=nz, **common) as c, \
            solver.Solver(nx=2 * nx, ny=2 * ny, nz=2 * nz, **common) as f:
        g = (1.0 / 27.0 + 0.01 * rng.standard_normal((27, nz, ny, nx))).astype(np.float32)
        phi = rng.uniform(-0.05, 1.05, (nz, ny, nx)).astype(np.float32)
        u = (0.02 * rng.standard_normal((3, nz, ny, nx))).astype(np.float32)
        c.init_fields(np.zeros(c.n, np.float32), np.zeros(3 * c.n, np.float32))
        c.set_state(g, phi, u)
        f.init_fields(np.zeros(f.n, np.float32), np.zeros(3 * f.n, np.float32))
        solver.prolong2_state(c, f)
        gf, phif, uf = f.get_state()
    for got, src in ((gf, g), (phif, phi), (uf, u)):
        ref = _prolong_reference(src, wall)
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
    # the fine sums are 8 times the coarse ones: phi, p* = sum g, and the first moment of u
    assert np.isclose(phif.astype(np.float64).sum(), 8 * phi.astype(np.float64).sum(), rtol=1e-6)
    assert np.isclose(gf.astype(np.float64).sum(), 8 * g.astype(np.float64).sum(), rtol=1e-6)
    assert np.allclose(uf.astype(np.float64).sum(axis=(1, 2, 3)), 8 * u.astype(np.float64).sum(axis=(1, 2, 3)),
                       rtol=1e-5, atol=1e-4)


def test_prolongation_rejects_mismatched_boxes():
    common = dict(rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.01, width=4.0, mobility=0.1)
    with solver.Solver(nx=8, ny=8, nz=8, **common) as c, solver.Solver(nx=16, ny=16, nz=12, **common) as f:
        c.init_fields(np.zeros(c.n, np.float32), np.zeros(3 * c.n, np.float32))
        f.init_fields(np.zeros(f.n, np.float32), np.zeros(3 * f.n, np.float32))
        with pytest.raises(solver.LbmError) as e:
            solver.prolong2_state(c, f)
        assert e.value.status == -1


def _network(scale_u, zero=False):
    net = solver.Network(32, 32, 32, seed=5)
    if zero:
        net.set_params(np.zeros(solver.load().lbm_cnn_num_params(), np.float32))
    norm = solver.LbmClosureNorm.make([0.5, 0.0, 0.0, 0.0, 0.0], [0.5, 0.02, 0.02, 0.02, 0.01],
                                      [0.01, scale_u, scale_u, scale_u])
    return net, norm


def test_failing_corrected_run_falls_back_to_the_fine_solver():
    """A velocity correction of several lattice units per application trips the max |u| check at
    the first check; the run restarts from its first checkpoint (the restricted initial state) on
    the fine grid.  Its final state equals that state prolonged and run by the fine solver."""
    col = inputs.collision_set(1, seed=5, L=64, R=10.0)[0]
    net, norm = _network(5.0)
    steps, check = 32, 8
    with net:
        record, final = closure.run_with_fallback(net, norm, col, coarse_steps=steps, check_every=check,
                                                  apply_every=8)
        with final:
            got = final.get_state()
            assert final.step_count == 2 * steps
            obs = final.observables()
    fb = record["fallback"]
    assert record["final"] == "fine" and fb is not None
    assert fb["detected_at"] == check and fb["restart_from"] == 0 and fb["fine_steps"] == 2 * steps
    assert any("max |u|" in r for r in record["checks"][-1]["failed"])
    assert obs["n_nonfinite"] == 0
    # the same path by hand: restriction of the fine initial state, prolongation, fine steps
    ens = solver.Ensemble([col.params()])
    phi, u, ps = col.fields()
    ens.init_fields(0, *(np.ascontiguousarray(a, np.float32) for a in (phi, u, ps)))
    p = col.coarse_params()
    with solver.Solver(**p) as c, solver.Solver(**col.params()) as f:
        c.init_fields(np.zeros(c.n, np.float32), np.zeros(3 * c.n, np.float32))
        ens.restrict_state(0, c)
        f.init_fields(np.zeros(f.n, np.float32), np.zeros(3 * f.n, np.float32))
        solver.prolong2_state(c, f)
        f.step(2 * steps)
        want = f.get_state()
    ens.close()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_healthy_corrected_run_needs_no_fallback():
    col = inputs.collision_set(1, seed=5, L=64, R=10.0)[0]
    net, norm = _network(0.5, zero=True)
    with net:
        record, final = closure.run_with_fallback(net, norm, col, coarse_steps=32, check_every=8, apply_every=8)
        with final:
            assert final.step_count == 32
    assert record["final"] == "coarse" and record["fallback"] is None
    assert [c["step"] for c in record["checks"]] == [8, 16, 24, 32]
    assert all(not c["failed"] for c in record["checks"])
