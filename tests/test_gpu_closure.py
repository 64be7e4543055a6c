"""Learned closure kernels against the FP64 reference network (oracle/closure_ref.py) and against
their plain definitions.

Element by element, link by link (test_every_operation_matches_its_definition_elementwise): the
library's BF16 inputs, FP32 pre-activations and FP32 loss gradients of every layer are read back
(lbm_cnn_get_layer) and each operation of the pass is checked at every element against its
definition in the library's operand precision, evaluated in FP64 on the same values, within the
rigorous bound of FP32 accumulation (closure_ref: layer_bound, activation_bound, input_grad_bound,
weight_grad_bound; the FP32 loss gradient bit for bit).  Those bounds are below a quarter of one
product term of a convolution, so one wrong neighbour, channel group or plane fails them; they run
at the closure's 64^3 grid and on a ragged 64 x 40 x 37 grid (partial column tiles, uneven z
chunks), on the tcgen05 kernel and the mma.sync kernel.  End to end, the output stays within the
propagated bound of forward_lib at every element.

Against the FP64 network itself (BF16 rounding of both operands, unit roundoff 2^-8 each, about
4e-3 per product, averaging down over the 27 x 32-term sums): relative L2 error of the output
2e-2; of the gradient of every layer 3e-2, with cosine similarity >= 0.999 to the reference
gradient (a wrong sign, transpose or offset would give cosines far below 1).
"""
import numpy as np
import pytest

from oracle import closure_ref as R
from paper_2501_00846_b300 import inputs, solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    solver.load()


def _random_case(nx=32, ny=6, nz=5, seed=0):
    rng = np.random.default_rng(seed)
    flat = np.empty(solver.load().lbm_cnn_num_params(), np.float32)
    o = 0
    for cout, cin in solver.CNN_LAYERS:
        n = cout * cin * 27
        flat[o:o + n] = rng.uniform(-1, 1, n) * np.sqrt(6.0 / (27 * (cin + cout)))
        o += n
        flat[o:o + cout] = rng.uniform(-0.2, 0.2, cout)
        o += cout
    x = rng.standard_normal((5, nz, ny, nx)).astype(np.float32)
    t = (0.3 * rng.standard_normal((4, nz, ny, nx))).astype(np.float32)
    return flat, x, t


def _positive_case(nx, ny, nz, seed=0):
    """Weights >= 0, biases > 0, inputs in [0, 1] and targets below the output: every activation,
    loss gradient and layer gradient is positive, so no sum cancels and the weight-gradient bounds
    are tight relative to the gradients themselves."""
    rng = np.random.default_rng(seed)
    flat = np.empty(solver.load().lbm_cnn_num_params(), np.float32)
    o = 0
    for cout, cin in solver.CNN_LAYERS:
        n = cout * cin * 27
        flat[o:o + n] = rng.uniform(0, 2.0 / (27 * cin), n)
        o += n
        flat[o:o + cout] = rng.uniform(0.05, 0.3, cout)
        o += cout
    x = rng.uniform(0, 1, (5, nz, ny, nx)).astype(np.float32)
    y64, _ = R.forward(solver.Network.split(flat.astype(np.float64)), x.astype(np.float64))
    t = (y64 - 0.5).astype(np.float32)
    return flat, x, t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_matches_the_fp64_reference():
    import torch
    nx, ny, nz = 32, 6, 5
    flat, x, _ = _random_case(nx, ny, nz)
    with solver.Network(nx, ny, nz) as net:
        net.set_params(flat)
        xd = torch.from_numpy(x).cuda().reshape(-1)
        yd = torch.empty(4 * net.n, device="cuda")
        net.forward(xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().reshape(4, nz, ny, nx)
    ref, _ = R.forward(solver.Network.split(flat.astype(np.float64)), x.astype(np.float64))
    err = _rel(y, ref)
    print(f"forward rel L2 error {err:.3e}")
    assert err < 2e-2


def test_gradients_match_the_fp64_reference():
    import torch
    nx, ny, nz = 32, 6, 5
    flat, x, t = _random_case(nx, ny, nz, seed=1)
    with solver.Network(nx, ny, nz) as net:
        net.set_params(flat)
        xd = torch.from_numpy(x).cuda().reshape(-1)
        td = torch.from_numpy(t).cuda().reshape(-1)
        loss = net.grad(xd, td)
        g = net.get_grads()
    ref_loss, ref = R.loss_and_grads(solver.Network.split(flat.astype(np.float64)), x.astype(np.float64),
                                     t.astype(np.float64))
    assert abs(loss / ref_loss - 1) < 2e-2
    for l, ((gw, gb), (rw, rb)) in enumerate(zip(solver.Network.split(g), ref)):
        a = np.concatenate([gw.ravel(), gb.ravel()])
        b = np.concatenate([rw.ravel(), rb.ravel()])
        err = _rel(a, b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        print(f"layer {l + 1}: gradient rel L2 error {err:.3e}, cosine {cos:.6f}")
        assert err < 3e-2 and cos > 0.999


def test_accumulated_gradients_add_up_and_adam_reduces_the_loss():
    import torch
    nx, ny, nz = 32, 4, 4
    flat, x, t = _random_case(nx, ny, nz, seed=2)
    with solver.Network(nx, ny, nz) as net:
        net.set_params(flat)
        xd = torch.from_numpy(x).cuda().reshape(-1)
        td = torch.from_numpy(t).cuda().reshape(-1)
        net.grad(xd, td)
        g1 = net.get_grads()
        net.grad(xd, td, accumulate=True)
        g2 = net.get_grads()
        assert np.allclose(g2, 2 * g1, rtol=1e-5, atol=1e-9)
        losses = []
        for _ in range(30):
            losses.append(net.grad(xd, td))
            net.adam_step(1e-3)
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]


def test_restriction_matches_its_definition():
    import torch
    rng = np.random.default_rng(3)
    nx, ny, nz = 8, 6, 4
    phi = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    u = rng.standard_normal((3, nz, ny, nx)).astype(np.float32) * 0.01
    p = rng.standard_normal((nz, ny, nx)).astype(np.float32) * 1e-3
    rho_l, rho_g = 1.0, 0.01
    out = torch.empty(6 * nx * ny * nz // 8, device="cuda")
    solver.restrict2(torch.from_numpy(phi).cuda().reshape(-1), torch.from_numpy(u).cuda().reshape(-1),
                     torch.from_numpy(p).cuda().reshape(-1), nx, ny, nz, rho_l, rho_g, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(6, nz // 2, ny // 2, nx // 2)
    blk = lambda a: a.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).astype(np.float64)
    rho = rho_g + phi.astype(np.float64) * (rho_l - rho_g)
    phic = blk(phi).mean(axis=(1, 3, 5))
    assert np.allclose(got[0], phic, rtol=1e-6, atol=1e-7)
    for a in range(3):
        uc = (blk(rho * u[a]).sum(axis=(1, 3, 5))) / blk(rho).sum(axis=(1, 3, 5))
        assert np.allclose(got[1 + a], uc, rtol=1e-5, atol=1e-9)
    pc = blk(p).mean(axis=(1, 3, 5))
    assert np.allclose(got[4], pc, rtol=1e-5, atol=1e-10)
    assert np.allclose(got[5], 3 * pc / (rho_g + phic * (rho_l - rho_g)), rtol=1e-5, atol=1e-9)


def _closure_box():
    wl = inputs.static_droplet(L=32, radius=8.0, noise=0.01, seed=5)
    return wl


def test_zero_network_leaves_the_state_unchanged_and_a_constant_shifts_phi_only():
    """A zero network leaves the state bit for bit.  A constant network shifts phi in the bulk and
    compensates inside the interfaces (sum phi kept); its uniform velocity output is all momentum,
    which the correction removes, so ubar and the populations' first moment stay as they were."""
    wl = _closure_box()
    norm = solver.LbmClosureNorm.make([0.5, 0, 0, 0, 0], [0.5, 0.01, 0.01, 0.01, 1e-3], [1e-3, 1e-3, 2e-3, 3e-3])
    with solver.from_workload(wl) as s, solver.Network(wl.nx, wl.ny, wl.nz, stream=s.stream) as net:
        s.step(3)
        g0, phi0, u0 = s.get_state()
        net.set_params(np.zeros(net.num_params, np.float32))
        solver.closure_apply(s, net, norm)
        g1, phi1, u1 = s.get_state()
        assert np.array_equal(g0, g1) and np.array_equal(phi0, phi1) and np.array_equal(u0, u1)
        flat = np.zeros(net.num_params, np.float32)
        flat[-4:] = [1.0, 1.0, -1.0, 2.0]
        net.set_params(flat)
        solver.closure_apply(s, net, norm)
        g2, phi2, u2 = s.get_state()
        s.step(2)                                   # the corrected state steps on
        assert s.observables()["n_nonfinite"] == 0
    # phi: the sum is unchanged and no node leaves [min(phi, 0), max(phi, 1)]
    assert abs(phi2.astype(np.float64).sum() - phi1.astype(np.float64).sum()) < 1e-6 * phi1.size
    assert (phi2 >= np.minimum(phi1, 0) - 1e-6).all() and (phi2 <= np.maximum(phi1, 1) + 1e-6).all()
    assert np.abs(phi2 - phi1).max() > 1e-4
    assert np.abs(u2 - u1).max() < 1e-9
    c = np.array([[k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1] for k in range(27)], np.float64)
    assert np.abs(g2.astype(np.float64).sum(0) - g1.astype(np.float64).sum(0)).max() < 1e-6
    for a in range(3):
        j1 = np.tensordot(c[:, a], g1.astype(np.float64), axes=1)
        j2 = np.tensordot(c[:, a], g2.astype(np.float64), axes=1)
        assert np.abs(j2 - j1).max() < 2e-7


def test_velocity_correction_follows_its_definition_and_adds_no_momentum():
    """With a random network: ubar changes by du = out_scale y minus its rho-weighted mean (y the
    network's output on the state's features, rho from phi before the correction), so the box
    gains no momentum, and the populations' first moment moves by exactly du."""
    import torch
    wl = _closure_box()
    norm = solver.LbmClosureNorm.make([0.5, 0, 0, 0, 0], [0.5, 0.01, 0.01, 0.01, 1e-3], [0.0, 1e-3, 2e-3, 3e-3])
    flat, _, _ = _random_case(wl.nx, wl.ny, wl.nz, seed=12)
    with solver.from_workload(wl) as s, solver.Network(wl.nx, wl.ny, wl.nz, stream=s.stream) as net:
        net.set_params(flat)
        s.step(3)
        g1, phi1, u1 = s.get_state()
        x = torch.empty(5 * s.n, device="cuda")
        y = torch.empty(4 * s.n, device="cuda")
        solver.closure_features(s, norm, x)
        net.forward(x, y)
        solver.closure_apply(s, net, norm)
        g2, phi2, u2 = s.get_state()
        torch.cuda.synchronize()
        y = y.cpu().numpy().astype(np.float64).reshape((4,) + phi1.shape)
    assert np.array_equal(phi1, phi2)                       # out_scale[0] = 0: no phi correction
    rho = wl.rho_g + phi1.astype(np.float64) * (wl.rho_l - wl.rho_g)
    c = np.array([[k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1] for k in range(27)], np.float64)
    for a in range(3):
        raw = norm.out_scale[a + 1] * y[a + 1]
        du = raw - (rho * raw).sum() / rho.sum()
        assert np.abs(raw).max() > 1e-4
        np.testing.assert_allclose(u2[a] - u1[a], du, atol=2e-8)
        assert abs((rho * (u2[a].astype(np.float64) - u1[a])).sum()) < 1e-6 * (rho * np.abs(du)).sum()
        j1 = np.tensordot(c[:, a], g1.astype(np.float64), axes=1)
        j2 = np.tensordot(c[:, a], g2.astype(np.float64), axes=1)
        np.testing.assert_allclose(j2 - j1, du, atol=2e-7)


def test_features_and_targets_follow_their_definitions():
    import torch
    wl = _closure_box()
    norm = solver.LbmClosureNorm.make([0.5, 0, 0, 0, 0.0], [0.5, 0.01, 0.02, 0.03, 1e-3], [1e-3, 2e-3, 3e-3, 4e-3])
    with solver.from_workload(wl) as s:
        s.step(4)
        phi, u, p = s.read_fields()
        x = torch.empty(5 * s.n, device="cuda")
        solver.closure_features(s, norm, x)
        ref = torch.from_numpy(np.concatenate([phi.reshape(1, -1) + 0.01, u.reshape(3, -1) - 0.002]).astype(
            np.float32)).cuda().reshape(-1)
        t = torch.empty(4 * s.n, device="cuda")
        solver.closure_target(s, ref, norm, t)
        torch.cuda.synchronize()
        x, t = x.cpu().numpy().reshape(5, -1), t.cpu().numpy().reshape(4, -1)
    fields = [phi.reshape(-1), u[0].reshape(-1), u[1].reshape(-1), u[2].reshape(-1), p.reshape(-1)]
    for c in range(5):
        want = (fields[c] - norm.in_shift[c]) / norm.in_scale[c]
        assert np.allclose(x[c], want, rtol=1e-5, atol=1e-5 * np.abs(want).max())
    assert np.allclose(t[0], 0.01 / 1e-3, rtol=1e-3)
    for a in range(3):
        assert np.allclose(t[1 + a], -0.002 / norm.out_scale[1 + a], rtol=1e-3)


def test_trained_closure_beats_the_plain_coarse_run():
    """The whole pipeline at a small size: 32 seeded collisions on a 64^3 fine grid (R = 10),
    10 pairs each, 10 epochs; then a held-out collision run on the 32^3 coarse grid with and
    without the phi correction after every step, against the restricted fine run.  The closure
    must cut the RMS error of phi by at least a third over 120 coarse steps and keep the run
    finite."""
    from paper_2501_00846_b300 import closure
    cols = inputs.collision_set(33, seed=3, L=64, R=10.0)
    norm = closure.estimate_norm(cols[:4], stride=24)
    X, T = closure.generate(cols[:32], snapshots=10, stride=24, batch=16, norm=norm)
    with solver.Network(32, 32, 32, seed=3) as net:
        hist = closure.train(net, X, T, epochs=10, lr=2e-3)
        del X, T
        applied = solver.LbmClosureNorm.make(norm.in_shift, norm.in_scale, [norm.out_scale[0], 0.0, 0.0, 0.0])
        res = closure.evaluate(net, applied, cols[32], coarse_steps=120, every=20)
    print("loss", hist[0], "->", hist[-1], "plain", res["plain"], "closure", res["closure"])
    assert hist[-1] < 0.5 * hist[0]
    assert np.isfinite(res["closure"]["phi_rms_mean"])
    assert res["ratio_phi"] < 0.67


def test_every_8_closure_corrects_phi_and_u():
    """The closure in the form that applies the velocity correction: one network predicting the
    8-step defect (targets 8 coarse steps after a restriction), applied once every 8 coarse
    steps with both its phi and its u outputs.  Same small pipeline as above (32 collisions on a
    64^3 fine grid, 32^3 coarse).  The held-out run must stay finite, cut the phi error by at least
    a third and leave a smaller u error than the plain coarse run; applying the u output must also
    give a smaller u error than the same network's phi correction alone."""
    from paper_2501_00846_b300 import closure
    cols = inputs.collision_set(33, seed=3, L=64, R=10.0)
    norm = closure.estimate_norm(cols[:4], stride=24, every=8)
    X, T = closure.generate(cols[:32], snapshots=10, stride=24, batch=16, norm=norm, every=8)
    with solver.Network(32, 32, 32, seed=3) as net:
        hist = closure.train(net, X, T, epochs=10, lr=2e-3)
        del X, T
        both = solver.LbmClosureNorm.make(norm.in_shift, norm.in_scale, list(norm.out_scale))
        phi_only = solver.LbmClosureNorm.make(norm.in_shift, norm.in_scale, [norm.out_scale[0], 0.0, 0.0, 0.0])
        res = closure.evaluate(net, both, cols[32], coarse_steps=120, every=20, apply_every=8)
        res_phi = closure.evaluate(net, phi_only, cols[32], coarse_steps=120, every=20, apply_every=8)
    print("loss", hist[0], "->", hist[-1], "phi and u:", res["ratio_phi"], res["ratio_u"], "phi only:",
          res_phi["ratio_phi"], res_phi["ratio_u"])
    assert hist[-1] < 0.5 * hist[0]
    assert np.isfinite(res["closure"]["phi_rms_mean"]) and np.isfinite(res["closure"]["u_rms_mean"])
    assert res["ratio_phi"] < 0.67
    assert res["ratio_u"] < 1.0
    assert res["ratio_u"] < res_phi["ratio_u"]


def test_network_rejects_widths_that_are_not_a_multiple_of_32():
    """The convolution tiles x by 32 nodes: other widths are refused at creation (LBM_ERR_ARG)."""
    for nx in (48, 16, 0):
        with pytest.raises(solver.LbmError) as e:
            solver.Network(nx, 20, 3)
        assert e.value.status == -1


@pytest.mark.parametrize("shape", [(64, 16, 8), (32, 6, 5), (32, 3, 2)], ids=["tiles", "ragged-y", "tiny"])
def test_convolution_kernels_agree(shape):
    """All three convolution kernels add the same BF16 products in the same FP32 order per output:
    for each z offset -1, 0, +1, each in-plane offset, each 16-channel chunk (kernel 0, tcgen05 with
    TMEM accumulators, reads each input plane once for all three z offsets, whose column blocks land
    in consecutive output planes' accumulators in that order).  So outputs and gradients are
    identical, bit for bit, across kernels, at tile-multiple, ragged and tiny grids."""
    import torch
    nx, ny, nz = shape
    flat, x, t = _random_case(nx, ny, nz, seed=4)
    out = []
    for kernel in (0, 1, 2):
        with solver.Network(nx, ny, nz) as net:
            net.set_conv_kernel(kernel)
            net.set_params(flat)
            xd = torch.from_numpy(x).cuda().reshape(-1)
            td = torch.from_numpy(t).cuda().reshape(-1)
            yd = torch.empty(4 * net.n, device="cuda")
            net.forward(xd, yd)
            net.grad(xd, td)
            torch.cuda.synchronize()
            out.append((yd.cpu().numpy(), net.get_grads()))
    assert np.array_equal(out[1][0], out[2][0])
    assert np.array_equal(out[1][1], out[2][1])
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("L", [32, 64])
def test_back_to_back_calls_match_the_ordinary_launches_and_training_is_reproducible(L):
    """The tensor-core convolutions are launched with programmatic dependent launch: each sets up
    and loads its weights while the previous kernel drains, then waits for it.  Forward passes
    issued back to back with no host synchronisation, on inputs still being written, must equal
    kernel 1 (ordinary launches) bit for bit; and with no atomics left in the gradient or in the
    correction's sums, two identical training runs (gradient, Adam step, forward) must give
    bit-identical parameters and outputs."""
    import torch

    def run(kernel, nfwd=8, nsteps=6):
        g = torch.Generator(device="cuda").manual_seed(11)
        with solver.Network(L, L, L, seed=5) as net:
            net.set_conv_kernel(kernel)
            n = net.n
            xs = [torch.randn(5 * n, device="cuda", generator=g) for _ in range(nfwd)]
            ts = [0.1 * torch.randn(4 * n, device="cuda", generator=g) for _ in range(nsteps)]
            ys = [torch.empty(4 * n, device="cuda") for _ in range(nfwd + nsteps)]
            for i in range(nfwd):
                net.forward(xs[i], ys[i])
            first = [y.clone() for y in ys[:nfwd]]
            for i in range(nsteps):
                net.grad(xs[i], ts[i])
                net.adam_step(1e-3)
                net.forward(xs[(i + 1) % nfwd], ys[nfwd + i])
            torch.cuda.synchronize()
            return ([y.cpu().numpy() for y in first], [y.cpu().numpy() for y in ys[nfwd:]], net.get_params())

    tc, tc2, mma = run(0), run(0), run(1)
    for a, b in zip(tc[0], mma[0]):
        assert np.array_equal(a, b)
    assert np.array_equal(tc[2], tc2[2])
    for a, b in zip(tc[1], tc2[1]):
        assert np.array_equal(a, b)
    assert np.array_equal(tc[2], mma[2])


def test_tensor_core_wait_expiry_is_reported_and_the_network_recovers():
    """The tensor-core convolution bounds every mbarrier wait.  The test hook makes the first wait
    of every such launch expire (on a barrier no MMA is committed to, before any MMA is issued):
    forward and grad return LBM_ERR_TIMEOUT, and once the hook is off the same network gives the
    same outputs and loss as before."""
    import torch
    with solver.Network(32, 32, 16, seed=5) as net:
        net.set_conv_kernel(0)
        x = torch.randn(5 * net.n, device="cuda")
        t = 0.1 * torch.randn(4 * net.n, device="cuda")
        y0 = torch.empty(4 * net.n, device="cuda")
        net.forward(x, y0)
        loss0 = net.grad(x, t)
        net.test_expire_wait(True)
        y = torch.empty_like(y0)
        with pytest.raises(solver.LbmError) as e:
            net.forward(x, y)
        assert e.value.status == -5
        with pytest.raises(solver.LbmError) as e:
            net.grad(x, t)
        assert e.value.status == -5
        net.test_expire_wait(False)
        net.forward(x, y)
        assert torch.equal(y, y0)
        assert net.grad(x, t) == loss0


def _dweight_chain(nx, ny, nz):
    """Most FP32 additions along one product's path in the weight-gradient kernel, for any z split:
    16 inside its MMA, at most 16 nz accumulations in its block (16 MMAs of a 32 x 8 column tile
    per plane, at most nz planes), and at most (column tiles x nz) block partials in the ordered
    reduction."""
    tiles = (nx // 32) * (-(-ny // 8))
    return 16 + 16 * nz + tiles * nz


@pytest.mark.parametrize("shape,kernel,positive", [
    ((64, 64, 64), 0, False), ((64, 64, 64), 0, True), ((64, 40, 37), 0, False), ((64, 40, 37), 1, False)],
    ids=["64cube-tcgen05", "64cube-tcgen05-positive", "ragged-tcgen05", "ragged-mma.sync"])
def test_every_operation_matches_its_definition_elementwise(shape, kernel, positive):
    import torch
    nx, ny, nz = shape
    flat, x, t = (_positive_case if positive else _random_case)(nx, ny, nz, seed=11)
    params = solver.Network.split(flat.astype(np.float64))
    with solver.Network(nx, ny, nz) as net:
        net.set_conv_kernel(kernel)
        net.set_params(flat)
        xd = torch.from_numpy(x).cuda().reshape(-1)
        td = torch.from_numpy(t).cuda().reshape(-1)
        yd = torch.empty(4 * net.n, device="cuda")
        net.forward(xd, yd)
        net.grad(xd, td)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().reshape(4, nz, ny, nx)
        grads = solver.Network.split(net.get_grads())
        layers = [net.get_layer(l) for l in range(4)]
    worst = check_against_definitions(params, x, t, y, grads, layers)
    y64, _ = R.forward(params, x.astype(np.float64))
    err = _rel(y, y64)
    print(f"{shape} kernel {kernel}{' positive' if positive else ''}: rel L2 vs FP64 {err:.2e}; "
          "largest |error| / bound: " + ", ".join(f"{k} {v:.2g}" for k, v in worst.items()))
    assert err < 2e-2


def check_against_definitions(params, x, t, y, grads, layers):
    """Every element of every operation of one forward and backward pass (the library's values y,
    grads [(dW, db)], layers [(a_in, z, dz)]) against its definition; returns the largest
    |error| / bound of each."""
    nz, ny, nx = x.shape[1:]
    worst = {}

    def within(name, got, ref, bound):
        ex = np.abs(np.asarray(got, np.float64) - ref) - bound
        assert (ex <= 0).all(), f"{name}: {int((ex > 0).sum())} elements outside the bound, worst excess {ex.max():.3e}"
        worst[name] = float((np.abs(np.asarray(got, np.float64) - ref) / np.maximum(bound, 1e-300)).max())

    assert np.array_equal(layers[0][0], R.bf16(x)), "layer-0 input is not bf16(x)"
    for l in range(4):
        a, z, _ = layers[l]
        zr, bz = R.layer_bound(*params[l], a)
        within(f"z{l}", z, zr, bz)
        if l < 3:
            r, ea = R.activation_bound(z)
            within(f"a{l + 1}", layers[l + 1][0], r, ea)
    assert np.array_equal(y, layers[3][1]), "output differs from the last pre-activation"
    assert np.array_equal(layers[3][2], R.loss_grad_fp32(layers[3][1], t)), "loss gradient is not the FP32 one"
    for l in range(3, 0, -1):
        ref, bz = R.input_grad_bound(params[l][0], layers[l][2], layers[l - 1][1])
        within(f"dz{l - 1}", layers[l - 1][2], ref, bz)
    n = nx * ny * nz
    for l in range(4):
        a, _, dz = layers[l]
        dW, bW = R.weight_grad_bound(dz, a, _dweight_chain(nx, ny, nz))
        within(f"dW{l}", grads[l][0], dW, bW)
        dz64 = dz.astype(np.float64)
        within(f"db{l}", grads[l][1], dz64.sum(axis=(1, 2, 3)), R.chain_gamma(n) * np.abs(dz64).sum(axis=(1, 2, 3)))
    fwd = R.forward_lib(params, x)
    within("y (end to end)", y, fwd[-1]["z"], fwd[-1]["D"])
    return worst


def test_on_policy_training_keeps_the_velocity_corrected_run_finite():
    """Trained on one-step pairs alone, the network's velocity correction drives the closed loop
    off the data it was trained on and the corrected run diverges within tens of steps.  Pairs
    collected along the corrected run's own short rollouts (closure.generate with a policy),
    added over two rounds of retraining, keep the run with phi and u both corrected finite over
    120 coarse steps, with phi still improved by at least a third."""
    from paper_2501_00846_b300 import closure
    cols = inputs.collision_set(33, seed=3, L=64, R=10.0)
    norm = closure.estimate_norm(cols[:4], stride=24)
    X, T = closure.generate(cols[:32], snapshots=10, stride=24, batch=16, norm=norm)
    Xs, Ts = [X], [T]
    with solver.Network(32, 32, 32, seed=3) as net:
        closure.train(net, X, T, epochs=10, lr=2e-3)
        for r in range(2):
            Xp, Tp = closure.generate(cols[:32], snapshots=10, stride=24, batch=16, norm=norm, policy=(net, norm),
                                      rollout=6, seed=r + 1)
            Xs.append(Xp)
            Ts.append(Tp)
            closure.train(net, Xs, Ts, epochs=10, lr=2e-3, seed=r + 1)
        del Xs, Ts
        res = closure.evaluate(net, norm, cols[32], coarse_steps=120, every=20)
    print("phi and u corrected, on-policy:", res["ratio_phi"], res["ratio_u"])
    assert np.isfinite(res["closure"]["phi_rms_mean"]) and np.isfinite(res["closure"]["u_rms_mean"])
    assert res["ratio_phi"] < 0.67
