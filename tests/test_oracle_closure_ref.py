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
