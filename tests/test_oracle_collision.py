"""Brute-force per-node pins of the oracle's kinetic building blocks.

Hermite tensors and moments are computed here from the lattice definition, independently of
the oracle's tables.  What each check pins (paper Section "High-order thread-safe LBM"):
  * f^eq (Eq. eqts) reproduces the Maxwellian moments p*, u, p* cs^2 d + uu and, for every
    third-order component the D3Q27 lattice supports, uuu;
  * S (Eq. guoforce, with F read as the acceleration a) has moments 0, a, ua + au;
  * f^neq (Eq. noneqts with weights, reading R7) has moments 0, 0, A, a3;
  * the collision obeys I1-I6: sum g = p*, sum g c = j + a, sum H2 g = uu + (1-w)A + (ua+au)/2,
    the literal-sum A equals its closed form, and on populations already in the Hermite span
    the regularised update equals Guo-forced BGK f - w (f - f^eq) + (1 - w/2) S.
"""
import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0
D = np.eye(3)


def _lattice():
    c = np.array([(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)],
                 dtype=np.float64)
    n2 = (c * c).sum(1)
    w = np.select([n2 == 0, n2 == 1, n2 == 2, n2 == 3], [8 / 27, 2 / 27, 1 / 54, 1 / 216])
    H2 = np.einsum("ia,ib->iab", c, c) - CS2 * D[None]
    H3 = (np.einsum("ia,ib,ig->iabg", c, c, c)
          - CS2 * (np.einsum("ia,bg->iabg", c, D) + np.einsum("ib,ag->iabg", c, D)
                   + np.einsum("ig,ab->iabg", c, D)))
    return c, w, H2, H3


C, W, H2, H3 = _lattice()
# third-order components the lattice supports: not all three indices equal
SUPPORTED = [(a, b, g) for a in range(3) for b in range(3) for g in range(3) if not (a == b == g)]


def _rand_state(rng):
    pstar = rng.normal(scale=0.05)
    u = rng.normal(scale=0.05, size=3)
    acc = rng.normal(scale=1e-3, size=3)
    A = rng.normal(scale=1e-3, size=(3, 3))
    A = 0.5 * (A + A.T)
    return pstar, u, acc, A


def test_equilibrium_moments():
    rng = np.random.default_rng(11)
    for _ in range(200):
        pstar, u, _, _ = _rand_state(rng)
        f = oracle.equilibrium(pstar, u)
        assert abs(f.sum() - pstar) < 1e-15
        np.testing.assert_allclose(C.T @ f, u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, C, C), pstar * CS2 * D + np.outer(u, u),
                                   atol=1e-15)
        m3 = np.einsum("i,iabg->abg", f, H3)
        for (a, b, g) in SUPPORTED:
            assert abs(m3[a, b, g] - u[a] * u[b] * u[g]) < 1e-15
        for a in range(3):
            assert abs(m3[a, a, a]) < 1e-15      # H3_aaa vanishes on D3Q27


def test_guo_source_moments():
    rng = np.random.default_rng(12)
    for _ in range(200):
        _, u, acc, _ = _rand_state(rng)
        S = oracle.guo_source(u, acc)
        assert abs(S.sum()) < 1e-16
        np.testing.assert_allclose(C.T @ S, acc, atol=1e-16)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", S, C, C),
                                   np.outer(u, acc) + np.outer(acc, u), atol=1e-16)


def test_nonequilibrium_moments():
    rng = np.random.default_rng(13)
    for _ in range(200):
        _, u, _, A = _rand_state(rng)
        fneq = oracle.nonequilibrium(A, u)
        assert abs(fneq.sum()) < 1e-16
        np.testing.assert_allclose(C.T @ fneq, 0, atol=1e-16)
        np.testing.assert_allclose(np.einsum("i,iab->ab", fneq, H2), A, atol=1e-16)
        a3 = (np.einsum("a,bg->abg", u, A) + np.einsum("b,ag->abg", u, A)
              + np.einsum("g,ab->abg", u, A))
        m3 = np.einsum("i,iabg->abg", fneq, H3)
        for (a, b, g) in SUPPORTED:
            assert abs(m3[a, b, g] - a3[a, b, g]) < 1e-16


def _random_populations(rng):
    pstar, u, acc, A = _rand_state(rng)
    f = W * (pstar + rng.normal(scale=0.02, size=27))
    return f, acc


def test_collision_invariants_I1_to_I5():
    rng = np.random.default_rng(14)
    for _ in range(3000):
        f, acc = _random_populations(rng)
        omega = rng.uniform(0.55, 1.95)
        g, u, A = oracle.collide_node(f, acc, omega)
        pstar = f.sum()
        j = C.T @ f
        Pi = np.einsum("i,ia,ib->ab", f, C, C)
        # Eq. moments1 with reading R1
        np.testing.assert_allclose(u, j + 0.5 * acc, atol=1e-16)
        # I5: closed form of Eq. hermite_neq2
        A_closed = Pi - CS2 * pstar * D - np.outer(u, u) + 0.5 * (np.outer(u, acc) + np.outer(acc, u))
        np.testing.assert_allclose(A, A_closed, atol=1e-15)
        # I1
        assert abs(g.sum() - pstar) < 1e-15
        # I2
        np.testing.assert_allclose(C.T @ g, j + acc, atol=1e-15)
        # I3
        expect = np.outer(u, u) + (1 - omega) * A + 0.5 * (np.outer(u, acc) + np.outer(acc, u))
        np.testing.assert_allclose(np.einsum("i,iab->ab", g, H2), expect, atol=1e-15)
        # third-order moment: uuu + (1 - w) a3 on the supported components
        a3 = (np.einsum("a,bg->abg", u, A) + np.einsum("b,ag->abg", u, A)
              + np.einsum("g,ab->abg", u, A))
        m3 = np.einsum("i,iabg->abg", g, H3)
        for (a, b, c) in SUPPORTED:
            assert abs(m3[a, b, c] - (u[a] * u[b] * u[c] + (1 - omega) * a3[a, b, c])) < 1e-15


def test_collision_I6_equals_guo_bgk_in_hermite_span():
    rng = np.random.default_rng(15)
    for _ in range(1000):
        pstar, u, acc, A = _rand_state(rng)
        omega = rng.uniform(0.55, 1.95)
        feq = oracle.equilibrium(pstar, u)
        S = oracle.guo_source(u, acc)
        f = feq - 0.5 * S + oracle.nonequilibrium(A, u)
        g, u_out, A_out = oracle.collide_node(f, acc, omega)
        np.testing.assert_allclose(u_out, u, atol=1e-16)
        np.testing.assert_allclose(A_out, A, atol=1e-16)
        bgk = f - omega * (f - feq) + (1 - 0.5 * omega) * S
        np.testing.assert_allclose(g, bgk, atol=1e-16)


def test_collision_at_rest_is_identity_on_equilibrium():
    """No force, populations at equilibrium: the collision returns them unchanged."""
    for pstar in (0.0, 0.3, -0.1):
        feq = oracle.equilibrium(pstar, np.zeros(3))
        g, u, A = oracle.collide_node(feq, np.zeros(3), 1.3)
        np.testing.assert_allclose(g, feq, atol=1e-17)
        np.testing.assert_allclose(u, 0, atol=1e-17)


def test_chemical_potential_vanishes_on_tanh_profile():
    """F^s = mu_phi grad(phi) with beta = 12 sigma/W, kappa = 3 sigma W/2 vanishes on the
    continuous equilibrium profile phi = 1/2 + 1/2 tanh(2x/W) (reading R9): there
    phi' = (4/W) phi (1-phi) and phi'' = (4/W)(1 - 2 phi) phi'."""
    P = oracle.Params(4, 4, 4, sigma=0.013, width=5.0, rho_l=1.0, rho_g=1.0, mu_l=0.1, mu_g=0.1)
    feq = oracle.equilibrium(0.0, np.zeros(3))
    for x in np.linspace(-8, 8, 41):
        phi = 0.5 + 0.5 * np.tanh(2 * x / P.width)
        d1 = 4 / P.width * phi * (1 - phi)
        d2 = 4 / P.width * (1 - 2 * phi) * d1
        F = oracle.force_node(P, feq, phi, np.array([d1, 0, 0]), d2, np.zeros(3))
        assert np.abs(F).max() < 1e-17
        # a profile of the wrong width is not at equilibrium
        F2 = oracle.force_node(P, feq, phi, np.array([d1, 0, 0]), 1.5 * d2, np.zeros(3))
        if 0.1 < phi < 0.4:
            assert np.abs(F2).max() > 1e-5


def test_viscous_force_relaxation_identity():
    """nu omega / cs^2 = 1 - omega/2 (tau = nu/cs^2 + 1/2): F^nu = -(1 - w/2) M grad(rho) with
    M = sum (f - f^eq(p*, ubar)) c c.  With sigma = 0, p* = 0 and no gravity only F^nu acts."""
    rng = np.random.default_rng(16)
    P = oracle.Params(4, 4, 4, sigma=0.0, rho_l=1.0, rho_g=0.01, mu_l=0.05, mu_g=0.002)
    for _ in range(100):
        phi = rng.uniform(0.05, 0.95)
        ubar = rng.normal(scale=0.03, size=3)
        M = rng.normal(scale=1e-3, size=(3, 3))
        M = 0.5 * (M + M.T)
        M -= np.trace(M) / 3 * D             # traceless so p* stays 0
        feq = oracle.equilibrium(0.0, ubar)
        f = feq + W * np.einsum("iab,ab->i", H2, M) / (2 * CS2 ** 2)
        gphi = rng.normal(size=3)
        F = oracle.force_node(P, f, phi, gphi, 0.0, ubar)
        rho = phi * P.rho_l + (1 - phi) * P.rho_g
        mu = phi * P.mu_l + (1 - phi) * P.mu_g
        omega = 1.0 / ((mu / rho) / CS2 + 0.5)
        grho = (P.rho_l - P.rho_g) * gphi
        np.testing.assert_allclose(F, -(1 - omega / 2) * M @ grho, rtol=1e-12, atol=1e-18)
