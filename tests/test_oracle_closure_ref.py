"""Pins of the FP64 closure-network reference (oracle/closure_ref.py): its convolution against
a direct sum and a pure shift, translation equivariance, and its analytic gradients against
central finite differences (so a wrong sign, index or transpose in the backward pass fails)."""
import numpy as np

from oracle import closure_ref as R


def _params(rng, scale=0.3):
    out = []
    for cin, cout in zip(R.CHANNELS[:-1], R.CHANNELS[1:]):
        out.append((rng.uniform(-scale, scale, (cout, cin, 27)) / np.sqrt(cin),
                    rng.uniform(-0.1, 0.1, cout)))
    return out


def test_offsets_follow_the_d3q27_index():
    assert R.OFFSETS[13] == (0, 0, 0)
    for k, (dz, dy, dx) in enumerate(R.OFFSETS):
        assert k == 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1)


def test_conv_equals_direct_sum_and_delta_kernel_is_a_shift():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((3, 4, 5, 6))
    W = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    z = R.conv(a, W, b)
    o, zz, yy, xx = 1, 3, 0, 5
    ref = b[o]
    for k, (dz, dy, dx) in enumerate(R.OFFSETS):
        for i in range(3):
            ref += W[o, i, k] * a[i, (zz + dz) % 4, (yy + dy) % 5, (xx + dx) % 6]
    assert abs(z[o, zz, yy, xx] - ref) < 1e-12
    D = np.zeros((3, 3, 27))
    for i in range(3):
        D[i, i, 9 * 2 + 3 * 1 + 0] = 1.0          # offset (dz, dy, dx) = (1, 0, -1)
    s = R.conv(a, D, np.zeros(3))
    assert np.array_equal(s, np.roll(a, shift=(-1, 0, 1), axis=(1, 2, 3)))


def test_network_is_translation_equivariant():
    rng = np.random.default_rng(1)
    p = _params(rng)
    x = rng.standard_normal((5, 4, 4, 6))
    y, _ = R.forward(p, x)
    ys, _ = R.forward(p, np.roll(x, shift=(1, 2, 3), axis=(1, 2, 3)))
    assert np.allclose(ys, np.roll(y, shift=(1, 2, 3), axis=(1, 2, 3)), atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    p = _params(rng)
    x = rng.standard_normal((5, 3, 4, 4))
    t = rng.standard_normal((4, 3, 4, 4)) * 0.1
    loss, grads = R.loss_and_grads(p, x, t)
    h = 1e-6
    for l in range(4):
        W, b = p[l]
        for _ in range(6):
            o, i, k = rng.integers(W.shape[0]), rng.integers(W.shape[1]), rng.integers(27)
            Wp, Wm = W.copy(), W.copy()
            Wp[o, i, k] += h
            Wm[o, i, k] -= h
            pp = list(p); pp[l] = (Wp, b)
            pm = list(p); pm[l] = (Wm, b)
            fd = (R.loss_and_grads(pp, x, t)[0] - R.loss_and_grads(pm, x, t)[0]) / (2 * h)
            assert abs(fd - grads[l][0][o, i, k]) <= 1e-6 * max(1.0, abs(fd)), (l, o, i, k, fd, grads[l][0][o, i, k])
        o = rng.integers(b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[o] += h
        bm[o] -= h
        pp = list(p); pp[l] = (W, bp)
        pm = list(p); pm[l] = (W, bm)
        fd = (R.loss_and_grads(pp, x, t)[0] - R.loss_and_grads(pm, x, t)[0]) / (2 * h)
        assert abs(fd - grads[l][1][o]) <= 1e-6 * max(1.0, abs(fd))


# ---- the library's operand precision and the rounding bounds --------------------------------------

def test_bf16_rounding_matches_torch_including_ties():
    """bf16() against torch's float32 -> bfloat16 conversion (round to nearest, ties to even) on
    random magnitudes, signs and exact midpoints between neighbouring bfloat16 values."""
    import torch
    rng = np.random.default_rng(7)
    v = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    # midpoints: 1 + (2j + 1) 2^-8 lies halfway between 1 + j 2^-7 and 1 + (j + 1) 2^-7
    j = np.arange(0, 128)
    mids = np.concatenate([1.0 + (2 * j + 1) * 2.0 ** -8, -(3.0 + (2 * j + 1) * 2.0 ** -7)]).astype(np.float32)
    for arr in (v, mids, np.array([0.0, -0.0, 1.0, 2.0 ** -20, 65504.0], np.float32)):
        want = torch.from_numpy(arr).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(R.bf16(arr), want)
    # ties go to the even significand: 1 + 2^-8 -> 1, 1 + 3 2^-8 -> 1 + 2^-6
    assert R.bf16(1.0 + 2.0 ** -8) == 1.0 and R.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def _emulated_layer(W, b, a_lib, plant=None):
    """The library's arithmetic for one layer on the CPU: BF16 weights and inputs, exact products,
    float32 sums (BLAS sgemm per offset, then float32 adds over the offsets and the bias).  plant:
    (k, node) whose neighbour value at offset k is replaced by the node's own value (a planted
    halo mistake)."""
    Wb = R.bf16(W).astype(np.float32)
    a = np.asarray(a_lib, np.float32)
    cin = a.shape[0]
    z = np.broadcast_to(np.asarray(b, np.float32)[:, None], (W.shape[0], a[0].size)).copy()
    for k, off in enumerate(R.OFFSETS):
        s = R.shifted(a, off).reshape(cin, -1).copy()
        if plant is not None and plant[0] == k:
            s[:, plant[1]] = a.reshape(cin, -1)[:, plant[1]]
        z += Wb[:, :, k] @ s
    return z.reshape((W.shape[0],) + a.shape[1:])


def _glorot(rng, positive=False):
    out = []
    for cin, cout in zip(R.CHANNELS[:-1], R.CHANNELS[1:]):
        lim = np.sqrt(6.0 / (27 * (cin + cout)))
        W = rng.uniform(-lim, lim, (cout, cin, 27))
        out.append((np.abs(W) if positive else W, rng.uniform(-0.2, 0.2, cout)))
    return out


def _silu32(z):
    z = np.asarray(z, np.float32)
    return z / (np.float32(1) + np.exp(-z))


def _silu_grad32(z):
    z = np.asarray(z, np.float32)
    s = np.float32(1) / (np.float32(1) + np.exp(-z))
    return s * (np.float32(1) + z * (np.float32(1) - s))


def test_library_precision_bounds_hold_for_float32_arithmetic():
    """The network evaluated as the library does it (emulated on the CPU: BF16 operands, float32
    sums in BLAS order, float32 silu and silu') satisfies every bound of the oracle, link by link on
    its own values (layer_bound, activation_bound, input_grad_bound, weight_grad_bound, the FP32 loss
    gradient) and end to end against forward_lib; the own-value bounds are tight: the accumulation
    bound of a convolution is below a quarter of the mean size of one of its product terms."""
    rng = np.random.default_rng(8)
    for trial in range(3):
        p = _glorot(rng, positive=trial == 2)
        x = rng.standard_normal((5, 6, 5, 8)).astype(np.float32)
        t = (0.3 * rng.standard_normal((4, 6, 5, 8))).astype(np.float32)
        fwd = R.forward_lib(p, x)
        a = R.bf16(x).astype(np.float32)
        acts, zs = [], []
        for l, (W, b) in enumerate(p):
            z = _emulated_layer(W, b, a)
            zr, bound = R.layer_bound(W, b, a)
            assert (np.abs(z - zr) <= bound).all(), (trial, l)
            S = R.conv(np.abs(a), np.abs(R.bf16(W)), np.abs(b))
            assert (bound <= 0.25 * S / R.conv_padded_chain(W.shape[1])).all()
            assert (np.abs(a - fwd[l]["a"]) <= fwd[l]["E"]).all() and (np.abs(z - fwd[l]["z"]) <= fwd[l]["D"]).all()
            acts.append(a)
            zs.append(z)
            a = R.bf16(_silu32(z)).astype(np.float32)
            r, eb = R.activation_bound(z)
            assert (np.abs(a - r) <= eb).all() and (eb == 0).mean() > 0.9
        dz = R.loss_grad_fp32(zs[3], t)
        n = x[0].size
        for l in range(3, -1, -1):
            dzb = R.bf16(dz).astype(np.float32)
            dW32 = np.empty((dz.shape[0], acts[l].shape[0], 27), np.float32)
            for k, off in enumerate(R.OFFSETS):
                dW32[:, :, k] = dzb.reshape(dz.shape[0], -1) @ R.shifted(acts[l], off).reshape(acts[l].shape[0], -1).T
            dW, bW = R.weight_grad_bound(dz, acts[l], chain=n)
            assert (np.abs(dW32 - dW) <= bW).all(), (trial, l)
            if l == 0:
                break
            Wb = R.bf16(p[l][0]).astype(np.float32)
            da = np.zeros((Wb.shape[1], n), np.float32)
            for k, off in enumerate(R.OFFSETS):
                da += Wb[:, :, k].T @ R.shifted(dzb, tuple(-o for o in off)).reshape(dz.shape[0], -1)
            dz_prev = da.reshape((Wb.shape[1],) + dz.shape[1:]) * _silu_grad32(zs[l - 1])
            ref, bz = R.input_grad_bound(p[l][0], dz, zs[l - 1])
            assert (np.abs(dz_prev - ref) <= bz).all(), (trial, l)
            dz = dz_prev


def test_layer_bound_accepts_the_library_arithmetic_and_catches_a_planted_halo_mistake():
    """layer_bound is tight enough that one wrong neighbour of one node (a staging or descriptor
    mistake at a tile edge) fails it, while float32 accumulation in any order passes."""
    rng = np.random.default_rng(9)
    W, b = _glorot(rng)[1]
    a = R.bf16(rng.standard_normal((32, 6, 5, 8)))
    zr, bound = R.layer_bound(W, b, a)
    z = _emulated_layer(W, b, a)
    assert (np.abs(z - zr) <= bound).all()
    node = 3 * 40 + 2 * 8 + 7                # x = 7: the +x neighbour wraps to x = 0
    zp = _emulated_layer(W, b, a, plant=(14, node))
    bad = np.abs(zp - zr) > bound
    assert bad.any() and bad.reshape(32, -1)[:, node].any()
