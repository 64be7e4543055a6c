"""Pins of the oracle's emulation of the library's 16-bit population storage (oracle.Params
storage16 = 1 BF16, 2 FP16), against the storage's definition rather than against the oracle.

The storage is the precision form of the populations (not in the paper): a node keeps
h_i = g_i / w_i - p* - e_i(u), rounded to BF16, or to FP16 after scaling by 2^12, plus
P = p* - sum_i w_i hr_i; it represents the populations w_i (P + e_i(u) + hr_i).  Here e_i(u) is
the third-order equilibrium without its p* part, written out independently of the oracle:
e_i = 3 cu + 4.5 cu^2 - 1.5 u^2 + 4.5 cu^3 - 4.5 cu u^2 (cu = c_i . u).  Checks:
  * per node (oracle.store16_node): hr is the FP32 deviation rounded by torch's BF16 conversion or
    numpy's float16 (independent rounding routines), P + sum w hr = p*, and the represented
    populations are w (P + e + hr);
  * over one oracle step of a noisy droplet: each node's sum of populations equals the unrounded
    step's (p* survives the rounding), and each population moves by at most
    w_i (|d_i| + sum_j w_j |d_j|), d the rounding of h (half a unit of the format at each h), with
    the rounding visible.
"""
import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs

UNIT = {1: 2.0 ** -8, 2: 2.0 ** -11}   # unit roundoff (half an ulp at 1) of BF16 and FP16


def _e(u):
    """e_i(u) [27, ...] = f^eq_i(0, u) / w_i of the third-order equilibrium."""
    c, _ = oracle.lattice()
    cu = np.einsum("ia,a...->i...", c.astype(np.float64), u)
    u2 = (u * u).sum(axis=0)
    return 3.0 * cu + 4.5 * cu * cu - 1.5 * u2 + 4.5 * cu ** 3 - 4.5 * cu * u2


def _one_step(storage16, L=12):
    wl = inputs.static_droplet(L=L, radius=3.0, noise=0.01, seed=7)
    P = oracle.Params(**wl.params(), storage16=storage16)
    ps = wl.pstar_init()
    s0 = oracle.init(P, wl.phi0(), wl.u0(), ps)
    return P, s0, oracle.step(P, s0)


def _deviation(s):
    _, w = oracle.lattice()
    wb = w.reshape((27,) + (1,) * 3)
    pstar = s.g.sum(axis=0)
    return s.g / wb - pstar[None] - _e(s.u), wb


@pytest.mark.parametrize("fmt", [1, 2], ids=["bf16", "fp16"])
def test_stored_pair_is_the_rounded_deviation_and_rebuilds_the_populations(fmt):
    """Per node (oracle.store16_node, on the post-collision populations of a noisy droplet):
    hr is h = g / w - p* - e(u) rounded from FP32 to the format (torch's BF16 conversion, numpy's
    float16 after the 2^12 scaling, both round to nearest even); P + sum w hr = p*; and the
    represented populations are w (P + e + hr)."""
    import torch
    _, _, s = _one_step(0)
    c, w = oracle.lattice()
    rng = np.random.default_rng(3)
    nodes = [tuple(rng.integers(0, n) for n in s.phi.shape) for _ in range(40)]
    for z, y, x in nodes:
        g, u = s.g[:, z, y, x], s.u[:, z, y, x]
        P, hr, gout = oracle.store16_node(fmt, g, u)
        e = _e(u.reshape(3, 1))[:, 0]
        h32 = (g / w - g.sum() - e).astype(np.float32)
        if fmt == 1:
            want = torch.from_numpy(h32).to(torch.bfloat16).to(torch.float32).numpy()
        else:
            want = (h32 * np.float32(4096.0)).astype(np.float16).astype(np.float32) / np.float32(4096.0)
        assert np.array_equal(hr, want.astype(np.float64))
        assert abs(P + (w * hr).sum() - g.sum()) <= 1e-15 * max(abs(g.sum()), 1.0)
        assert np.allclose(gout, w * (P + e + hr), rtol=0, atol=1e-16)
        assert np.count_nonzero(hr) > 20                      # real deviations were rounded


@pytest.mark.parametrize("fmt", [1, 2], ids=["bf16", "fp16"])
def test_rounding_keeps_pstar_and_moves_populations_within_the_bound(fmt):
    P, s0, s16 = _one_step(fmt)
    P0 = oracle.Params(**{k: getattr(P, k) for k in P.__dataclass_fields__ if k != "storage16"})
    s = oracle.step(P0, s0)
    # p* per node: the storage rounds deviations whose weighted sum it returns through P
    ps, ps16 = s.g.sum(axis=0), s16.g.sum(axis=0)
    assert np.abs(ps16 - ps).max() <= 1e-13 * max(np.abs(ps).max(), 1.0)
    # each population: w_i (d_i - sum_j w_j d_j), |d| <= u16 |h| (+ the FP32 step before rounding)
    h, wb = _deviation(s)
    d = UNIT[fmt] * np.abs(h) + 2.0 ** -24 * np.abs(h) + 1e-300
    bound = wb * (d + (wb * d).sum(axis=0)[None])
    err = np.abs(s16.g - s.g)
    print(f"fmt {fmt}: largest |change| / bound {(err / bound).max():.3f}")
    assert (err <= bound * (1 + 1e-9) + 1e-15).all()
    assert err.max() > 0.05 * bound.max()                # the rounding is seen
    # the state apart from the populations is the unrounded step's
    assert np.array_equal(s16.phi, s.phi) and np.array_equal(s16.u, s.u)


# -- the 16-bit moment storage (storage16 = 3 BF16, 4 FP16) -------------------------------------

def _round_like_library(fmt, v):
    """FP32 value of v rounded to the format (torch's BF16 conversion; numpy's float16 of 2^12 v)."""
    import torch
    v32 = np.asarray(v, np.float32)
    if fmt == 1:
        return torch.from_numpy(v32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    return ((v32 * np.float32(4096.0)).astype(np.float16).astype(np.float32) / np.float32(4096.0)).astype(np.float64)


def test_moment_set_rebuilds_the_collided_populations():
    """The moment storage's set of a collided node, extracted by the moment identities (sum g = p*,
    sum g c = u + a/2, sum g c c = p* I/3 + (2/9)(B + 4.5 u u + 4.5 sym(u a))), is a = F / rho and
    B = 4.5 (1 - omega) A of the collision, and its polynomial gives back the collided populations:
    random pre-collision states, accelerations and relaxation rates, 200 nodes."""
    rng = np.random.default_rng(17)
    for _ in range(200):
        f = 1.0 / 27.0 + 0.02 * rng.standard_normal(27)
        acc = 0.002 * rng.standard_normal(3)
        omega = rng.uniform(0.5, 1.95)
        g, u, A = oracle.collide_node(f, acc, omega)
        ps, a, B = oracle.mom_extract(g, u)
        assert abs(ps - g.sum()) <= 1e-15
        assert np.abs(a - acc).max() <= 1e-14
        assert np.abs(B - 4.5 * (1.0 - omega) * A).max() <= 1e-14
        assert np.abs(oracle.mom_rebuild(ps, u, a, B) - g).max() <= 1e-15


@pytest.mark.parametrize("fmt", [1, 2], ids=["bf16", "fp16"])
def test_moment_storage_rounds_a_and_b_and_keeps_the_other_moments(fmt):
    """Per node of a stepped noisy droplet (oracle.store_mom16_node): the kept a and B are their
    FP32 values rounded by an independent routine; the represented populations keep p* and carry
    u + a_r / 2 as first moment, with a_r the rounded a."""
    _, _, s = _one_step(0)
    c, w = oracle.lattice()
    rng = np.random.default_rng(5)
    seen = 0
    for _ in range(40):
        z, y, x = (int(rng.integers(0, n)) for n in s.phi.shape)
        g, u = s.g[:, z, y, x], s.u[:, z, y, x]
        ps, a, B = oracle.mom_extract(g, u)
        ab, gout = oracle.store_mom16_node(fmt, g, u)
        want = np.concatenate([a, [B[0, 0], B[1, 1], B[2, 2], B[0, 1], B[0, 2], B[1, 2]]])
        assert np.array_equal(ab, _round_like_library(fmt, want))
        assert abs(gout.sum() - ps) <= 1e-15 * max(abs(ps), 1.0)
        assert np.abs(gout @ c.astype(np.float64) - (u + 0.5 * ab[:3])).max() <= 1e-15
        seen += np.count_nonzero(ab != want)
    assert seen > 100                                     # real moments were rounded


@pytest.mark.parametrize("fmt", [1, 2], ids=["bf16", "fp16"])
def test_moment_storage_step_keeps_pstar_and_fields(fmt):
    """One oracle step with the emulated moment storage: every node keeps the unrounded step's p*;
    phi and u are the unrounded step's; the populations differ, by about the format's rounding."""
    P, s0, s16 = _one_step(fmt + 2)
    P0 = oracle.Params(**{k: getattr(P, k) for k in P.__dataclass_fields__ if k != "storage16"})
    s = oracle.step(P0, s0)
    ps, ps16 = s.g.sum(axis=0), s16.g.sum(axis=0)
    assert np.abs(ps16 - ps).max() <= 1e-13 * max(np.abs(ps).max(), 1.0)
    assert np.array_equal(s16.phi, s.phi) and np.array_equal(s16.u, s.u)
    err = np.abs(s16.g - s.g).max()
    assert 0 < err <= 50 * UNIT[fmt] * np.abs(s.g - s.g.mean(axis=(1, 2, 3), keepdims=True)).max()
