"""FP64 reference of the learned closure's network (test infrastructure, like the rest of oracle/).

The paper has no learned component; the closure is this project's own addition (a coarse-grid
correction measured against the fine-grid solver).  This module is the plain, slow, obviously
correct definition that the GPU kernels' forward pass and gradients are checked against.  It is
never imported by the CUDA path.

Network (all layers periodic 3x3x3 convolutions on an nz x ny x nx grid):
    a_0 = x                                   (C_0 = 5 input channels)
    z_l[o, n] = b_l[o] + sum_{i, k} W_l[o, i, k] a_{l-1}[i, n + off_k]     l = 1..4
    a_l = silu(z_l) = z_l / (1 + exp(-z_l))   l = 1..3;    y = z_4        (C_4 = 4 outputs)
with channel counts 5, 32, 32, 32, 4, offsets off_k = (dz, dy, dx) for k = 9 (dz+1) + 3 (dy+1) +
(dx+1) (the D3Q27 index order), and n + off_k taken periodically.  Loss: mean over outputs and
nodes of (y - t)^2.
"""
import numpy as np

CHANNELS = (5, 32, 32, 32, 4)
OFFSETS = [(k // 9 - 1, (k // 3) % 3 - 1, k % 3 - 1) for k in range(27)]   # (dz, dy, dx)


def shifted(a, off):
    """a[c, z + dz, y + dy, x + dx] with periodic wrap (a: [C, nz, ny, nx])."""
    dz, dy, dx = off
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(1, 2, 3))


def conv(a, W, b):
    """z[o] = b[o] + sum_{i,k} W[o, i, k] a[i](n + off_k); W: [Cout, Cin, 27]."""
    z = np.empty((W.shape[0],) + a.shape[1:], np.float64)
    z[:] = b[:, None, None, None]
    for k, off in enumerate(OFFSETS):
        s = shifted(a, off)
        z += np.einsum("oi,izyx->ozyx", W[:, :, k], s)
    return z


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x):
    """params: list of (W, b) per layer; x: [5, nz, ny, nx].  Returns (y, cache)."""
    a = np.asarray(x, np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        z = conv(a, np.asarray(W, np.float64), np.asarray(b, np.float64))
        cache.append((a, z))
        a = silu(z) if l < len(params) - 1 else z
    return a, cache


def loss_and_grads(params, x, t):
    """Mean-squared loss and its gradients with respect to every W and b (backward pass written
    out: dz_L = 2 (y - t) / M; dW_l[o, i, k] = sum_n dz_l[o, n] a_{l-1}[i, n + off_k];
    db_l = sum_n dz_l; da_{l-1}[i, n] = sum_{o,k} W_l[o, i, k] dz_l[o, n - off_k];
    dz_{l-1} = da_{l-1} silu'(z_{l-1}))."""
    y, cache = forward(params, x)
    t = np.asarray(t, np.float64)
    M = y.size
    loss = float(((y - t) ** 2).mean())
    dz = 2.0 * (y - t) / M
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], np.float64)
        a_prev, _ = cache[l]
        dW = np.empty_like(W)
        for k, off in enumerate(OFFSETS):
            dW[:, :, k] = np.einsum("ozyx,izyx->oi", dz, shifted(a_prev, off))
        db = dz.sum(axis=(1, 2, 3))
        grads[l] = (dW, db)
        if l > 0:
            da = np.zeros_like(a_prev)
            for k, off in enumerate(OFFSETS):
                back = shifted(dz, tuple(-o for o in off))
                da += np.einsum("oi,ozyx->izyx", W[:, :, k], back)
            dz = da * silu_grad(cache[l - 1][1])
    return loss, grads
