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
    """z[o] = b[o] + sum_{i,k} W[o, i, k] a[i](n + off_k); W: [Cout, Cin, 27].  Each offset's
    channel contraction is one matrix product (BLAS) over all nodes."""
    cin = a.shape[0]
    z = np.empty((W.shape[0], a[0].size), np.float64)
    z[:] = np.asarray(b, np.float64)[:, None]
    for k, off in enumerate(OFFSETS):
        z += W[:, :, k] @ shifted(a, off).reshape(cin, -1)
    return z.reshape((W.shape[0],) + a.shape[1:])


def conv_transpose(d, W):
    """da[i, n] = sum_{o,k} W[o, i, k] d[o](n - off_k): the input gradient of conv."""
    cout = d.shape[0]
    da = np.zeros((W.shape[1], d[0].size), np.float64)
    for k, off in enumerate(OFFSETS):
        da += W[:, :, k].T @ shifted(d, tuple(-o for o in off)).reshape(cout, -1)
    return da.reshape((W.shape[1],) + d.shape[1:])


def weight_grad(dz, a):
    """dW[o, i, k] = sum_n dz[o, n] a[i](n + off_k): the weight gradient of conv."""
    cout, cin = dz.shape[0], a.shape[0]
    dW = np.empty((cout, cin, 27), np.float64)
    d2 = dz.reshape(cout, -1)
    for k, off in enumerate(OFFSETS):
        dW[:, :, k] = d2 @ shifted(a, off).reshape(cin, -1).T
    return dW


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
        dW = weight_grad(dz, a_prev)
        db = dz.sum(axis=(1, 2, 3))
        grads[l] = (dW, db)
        if l > 0:
            da = conv_transpose(dz, W)
            dz = da * silu_grad(cache[l - 1][1])
    return loss, grads


# ---- the network in the library's operand precision, and bounds on its rounding ----------------
#
# The library evaluates the same network with BF16 weights and BF16 layer inputs (the network input
# x and every silu(z) are rounded to BF16 before the next convolution reads them), exact products
# and FP32 accumulation, and keeps z, the loss gradient and the backward pass in FP32 (each
# backward convolution again reads BF16 operands).  The functions below give that rounding as a
# definition (bf16) and first-order bounds on how far it can move each value from the FP64
# network above.  Sums of FP32 numbers are bounded for any order of the additions, allowing each
# addition an error of one FP32 ulp (2 u32 relative) rather than half of one, so that tensor-core
# accumulators that truncate are covered too.

U_BF16 = 2.0 ** -8          # unit roundoff of bfloat16: 8 significant bits, round to nearest
U_FP32 = 2.0 ** -24         # unit roundoff of float32
SILU_LIP = 1.0999           # sup |silu'(z)| (1.09984 near z = 2.3994)
SILU2_MAX = 0.5             # sup |silu''(z)| (at z = 0)
EPS_ACT = 2.0 ** -19        # allowance for the FP32 evaluation of silu and silu' (relative)


def bf16(v):
    """v rounded to the nearest bfloat16 value (ties to even), as float64.  With v = m 2^e,
    1/2 <= |m| < 1, the 8 significant bits are round(m 2^8) (numpy rounds halves to even);
    bfloat16 has float32's exponent range, far from the values here."""
    m, e = np.frexp(np.asarray(v, np.float64))
    return np.ldexp(np.round(np.ldexp(m, 8)), e - 8)


def chain_gamma(n):
    """Bound factor of an FP32 sum of n + 1 terms in any order: |fl(sum) - sum| <= gamma sum |t|,
    with each of the n additions off by at most one ulp (first order)."""
    return n * 2.0 * U_FP32


def conv_padded_chain(cin):
    """Additions per output of the library's convolution: 27 offsets x the input channels padded
    to a multiple of 16 (the padded channels add zeros), plus the bias."""
    return 27 * (-(-cin // 16) * 16) + 1


def act_eps(z):
    """Relative error allowed for the library's FP32 silu(z) = z / (1 + e^-z) with a fast
    exponential whose relative error grows with |z|: that error reaches silu only through the share
    e^-z / (1 + e^-z) = 1 - sigmoid(z) of the denominator, so the allowance is
    (6 + (4 + 2 |z|) (1 - sigmoid(z))) float32 ulps (a generous one)."""
    z = np.asarray(z, np.float64)
    return (6.0 + (4.0 + 2.0 * np.abs(z)) * (1.0 - 1.0 / (1.0 + np.exp(-z)))) * 2.0 ** -23


def silu_grad_err(z):
    """Absolute error allowed for the library's FP32 silu'(z) = s (1 + z (1 - s)), s = sigmoid(z):
    the error of s (as in act_eps) times |d silu'/d s| <= 1 + 2 |z|, plus the rounding of the two
    products."""
    z = np.asarray(z, np.float64)
    s = 1.0 / (1.0 + np.exp(-z))
    return act_eps(z) * (1.0 + 2.0 * np.abs(z)) * s + 4.0 * U_FP32 * np.abs(silu_grad(z))


def _flip_bound(v, r, P):
    """Bound on |bf16(v') - r|, r = bf16(v), for any v' with |v' - v| <= P: rounding is monotone,
    so bf16(v') lies between bf16(v - P) and bf16(v + P); zero where both round to r."""
    return np.maximum(np.abs(bf16(v + P) - r), np.abs(r - bf16(v - P)))


def forward_lib(params, x):
    """The network in the library's operand precision with FP64 sums, and rigorous bounds on how
    far the library's FP32 evaluation can be from it.  Layer l reads a_l = bf16(x) (l = 0) or
    bf16(silu(z_{l-1})) and computes z_l = b_l + conv(a_l, bf16(W_l)) exactly; the library's z_l
    differs by its FP32 accumulation, gamma (|b| + conv(|a| + E, |W_b|)), plus the effect of inputs
    that rounded to the other neighbouring BF16 value, conv(E, |W_b|), where E bounds |a_lib - a|:
    zero unless the library's pre-rounding value, within P = SILU_LIP D (1 + eps) + eps |silu(z)|
    of silu(z), can lie across a rounding midpoint.  Returns a list of per-layer dicts with keys
    a, E (input and its bound), z, D (pre-activation and its bound)."""
    a = bf16(x)
    E = np.zeros_like(a)
    out = []
    nl = len(params)
    for l, (W, b) in enumerate(params):
        W = np.asarray(W, np.float64)
        b = np.asarray(b, np.float64)
        Wb = bf16(W)
        g = chain_gamma(conv_padded_chain(W.shape[1]))
        zero = np.zeros(W.shape[0])
        z = conv(a, Wb, b)
        D = g * (np.abs(b)[:, None, None, None] + conv(np.abs(a) + E, np.abs(Wb), zero)) + conv(E, np.abs(Wb), zero)
        out.append({"a": a, "E": E, "z": z, "D": D})
        if l == nl - 1:
            return out
        sv = silu(z)
        P = SILU_LIP * D * (1.0 + act_eps(z)) + act_eps(z) * np.abs(sv)
        a = bf16(sv)
        E = _flip_bound(sv, a, P)


def loss_grad_fp32(z3, t):
    """The library's loss gradient in FP32, operation by operation: scale = 2 / (4 N) and
    dz = scale (z - t), every operation rounded to float32 (z3 and t float32 [4][...])."""
    z3 = np.asarray(z3, np.float32)
    t = np.asarray(t, np.float32)
    scale = np.float32(2.0) / (np.float32(4.0) * np.float32(z3[0].size))
    return scale * (z3 - t)


def layer_bound(W, b, a_lib):
    """One forward convolution on the library's own BF16 input a_lib: the FP64 value its FP32
    accumulation approximates, z = b + conv(a_lib, bf16(W)) (a product of two BF16 numbers is exact
    in FP32 and FP64), and the bound gamma (|b| + conv(|a_lib|, |bf16(W)|)) on that accumulation's
    error.  Returns (z, bound)."""
    W = np.asarray(W, np.float64)
    b = np.asarray(b, np.float64)
    Wb = bf16(W)
    a = np.asarray(a_lib, np.float64)
    g = chain_gamma(conv_padded_chain(W.shape[1]))
    z = conv(a, Wb, b)
    bound = g * (np.abs(b)[:, None, None, None] + conv(np.abs(a), np.abs(Wb), np.zeros(W.shape[0])))
    return z, bound


def activation_bound(z_lib):
    """The next layer's input from the library's own FP32 pre-activation: r = bf16(silu(z_lib)), and
    the bound on |a_lib - r| left by the FP32 evaluation of silu (zero unless that evaluation, within
    act_eps of silu(z), can fall on the other side of a BF16 rounding midpoint).  Returns (r, bound)."""
    z = np.asarray(z_lib, np.float64)
    sv = silu(z)
    r = bf16(sv)
    return r, _flip_bound(sv, r, act_eps(z) * np.abs(sv))


def input_grad_bound(W, dz_lib, z_prev_lib):
    """The backward step through layer l on the library's own FP32 values: dz_{l-1} =
    conv_transpose(bf16(dz_l), bf16(W_l)) silu'(z_{l-1}), and the bound on the library's FP32
    evaluation (accumulation of the transposed convolution, FP32 silu', the final product).
    Returns (dz_prev, bound)."""
    W = np.asarray(W, np.float64)
    Wb = bf16(W)
    dzb = bf16(dz_lib)
    zp = np.asarray(z_prev_lib, np.float64)
    g = chain_gamma(conv_padded_chain(W.shape[0]))
    da = conv_transpose(dzb, Wb)
    Dda = g * conv_transpose(np.abs(dzb), np.abs(Wb))
    sg = silu_grad(zp)
    esg = silu_grad_err(zp)
    dz = da * sg
    return dz, Dda * (np.abs(sg) + esg) + np.abs(da) * esg + U_FP32 * (np.abs(dz) + Dda * (np.abs(sg) + esg))


def weight_grad_bound(dz_lib, a_lib, chain):
    """The weight gradient on the library's own values: dW = weight_grad(bf16(dz_lib), a_lib) and the
    bound chain_gamma(chain) weight_grad(|bf16(dz_lib)|, |a_lib|) for FP32 sums with at most `chain`
    additions along any term's path.  Returns (dW, bound)."""
    dzb = bf16(dz_lib)
    a = np.asarray(a_lib, np.float64)
    return weight_grad(dzb, a), chain_gamma(chain) * weight_grad(np.abs(dzb), np.abs(a))
