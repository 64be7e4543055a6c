"""Pins of the oracle's lattice tables and finite-difference stencils against closed forms.

The D3Q27 weights factorise, w(c) = w1(cx) w1(cy) w1(cz) with w1(0) = 2/3, w1(+-1) = 1/6, so
the isotropic stencils of the paper (Section "Model extension", gradient and Laplacian
formulas; Laplacian read as (2/cs^2) sum_{i!=0} w_i (psi(x+c_i) - psi(x))) have exact Fourier
symbols:
    G_a[e^{ik.x}] = i sin(k_a) prod_{b != a} (2 + cos k_b)/3 * e^{ik.x}
    L[e^{ik.x}]   = 6 (prod_b (2 + cos k_b)/3 - 1) e^{ik.x}
These are derived from the lattice definition, not from the oracle's code.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0


def _lattice_from_definition():
    c = np.array([(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)])
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
    w = np.array([w1[a] * w1[b] * w1[d] for a, b, d in c])
    return c, w


def test_lattice_matches_definition():
    c, w = oracle.lattice()
    c_ref, w_ref = _lattice_from_definition()
    assert np.array_equal(c, c_ref)
    np.testing.assert_allclose(w, w_ref, rtol=0, atol=1e-16)
    # rest vector and opposite pairs
    assert not c[13].any()
    for i in range(27):
        assert np.array_equal(c[26 - i], -c[i])


def test_lattice_isotropy():
    c, w = oracle.lattice()
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * d, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ig->abg", w, c, c, c), 0, atol=1e-16)
    four = np.einsum("i,ia,ib,ig,id->abgd", w, c, c, c, c)
    iso4 = CS2 ** 2 * (np.einsum("ab,gd->abgd", d, d) + np.einsum("ag,bd->abgd", d, d)
                       + np.einsum("ad,bg->abgd", d, d))
    np.testing.assert_allclose(four, iso4, atol=1e-16)


def _trig_field(P, k, theta):
    z, y, x = np.meshgrid(np.arange(P.nz), np.arange(P.ny), np.arange(P.nx), indexing="ij")
    arg = k[0] * x + k[1] * y + k[2] * z + theta
    return np.cos(arg), np.sin(arg)


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 2, 1), (3, -1, 2), (5, 4, -6)])
def test_gradient_and_laplacian_fourier_symbols(m):
    P = oracle.Params(12, 10, 14)
    k = 2 * math.pi * np.array(m) / np.array([P.nx, P.ny, P.nz])
    cosf, sinf = _trig_field(P, k, 0.3)
    g = oracle.grad(P, cosf)
    facs = (2.0 + np.cos(k)) / 3.0
    for a in range(3):
        other = np.prod([facs[b] for b in range(3) if b != a])
        np.testing.assert_allclose(g[a], -np.sin(k[a]) * other * sinf, atol=1e-13)
    lap = oracle.lap(P, cosf)
    np.testing.assert_allclose(lap, 6.0 * (np.prod(facs) - 1.0) * cosf, atol=1e-13)
    V = np.stack([cosf, 2 * cosf, -cosf])
    dv = oracle.div(P, V)
    expect = sum(-np.sin(k[a]) * np.prod([facs[b] for b in range(3) if b != a]) * sinf * s
                 for a, s in zip(range(3), (1, 2, -1)))
    np.testing.assert_allclose(dv, expect, atol=1e-13)


def test_polynomial_exactness_interior():
    """G is exact on linear fields, L on quadratic fields (checked away from the wrap)."""
    P = oracle.Params(9, 9, 9)
    z, y, x = np.meshgrid(np.arange(9.0), np.arange(9.0), np.arange(9.0), indexing="ij")
    lin = 0.7 * x - 1.3 * y + 0.25 * z + 2.0
    quad = x * x + 2 * y * y - z * z + 0.5 * x * y - 3 * y * z + x
    g = oracle.grad(P, lin)
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(g[0][inner], 0.7, atol=1e-12)
    np.testing.assert_allclose(g[1][inner], -1.3, atol=1e-12)
    np.testing.assert_allclose(g[2][inner], 0.25, atol=1e-12)
    L = oracle.lap(P, quad)
    np.testing.assert_allclose(L[inner], 2 + 4 - 2, atol=1e-11)
    gq = oracle.grad(P, quad)
    np.testing.assert_allclose(gq[0][inner], (2 * x + 0.5 * y + 1)[inner], atol=1e-11)
    np.testing.assert_allclose(gq[2][inner], (-2 * z - 3 * y)[inner], atol=1e-11)


def test_wall_extension_is_mirror():
    """With z walls the scalar field is extended evenly about z = -1/2 and z = nz - 1/2: the
    stencils then equal those of the periodic field on the doubled (mirrored) domain."""
    rng = np.random.default_rng(5)
    nx, ny, nz = 6, 5, 7
    phi = rng.random((nz, ny, nx))
    Pw = oracle.Params(nx, ny, nz, wall_z=1)
    Pp = oracle.Params(nx, ny, 2 * nz)
    doubled = np.concatenate([phi, phi[::-1]], axis=0)
    np.testing.assert_allclose(oracle.lap(Pw, phi), oracle.lap(Pp, doubled)[:nz], atol=1e-14)
    np.testing.assert_allclose(oracle.grad(Pw, phi), oracle.grad(Pp, doubled)[:, :nz], atol=1e-14)
    # vector: z component odd under the mirror
    V = rng.random((3, nz, ny, nx))
    Vd = np.concatenate([V, V[:, ::-1]], axis=1)
    Vd[2, nz:] *= -1
    np.testing.assert_allclose(oracle.div(Pw, V), oracle.div(Pp, Vd)[:nz], atol=1e-14)


@pytest.mark.parametrize("wall", [0, 1])
def test_stencils_telescope(wall):
    """Sum over the domain of L[psi] and div[V] vanish (periodic, and with the mirror walls):
    the property that makes the Allen-Cahn update conserve sum(phi)."""
    rng = np.random.default_rng(7 + wall)
    P = oracle.Params(7, 6, 8, wall_z=wall)
    psi = rng.random(P.shape)
    V = rng.normal(size=(3,) + P.shape)
    assert abs(oracle.lap(P, psi).sum()) < 1e-12
    assert abs(oracle.div(P, V).sum()) < 1e-12
