"""The identities behind moment-only storage, checked on the FP64 oracle's collision (no GPU).

Moment storage keeps, per node, p*, u, the acceleration a = F / rho and B = 4.5 (1 - omega) A
(A the regularised second-order non-equilibrium moment), and rebuilds each post-collision
population as the polynomial
    g_i / w_i = K0 + 4.5 cu (cu + ca) + cBc + cu (K1 + 4.5 cu^2 + 3 cBc) + c.v,
    K0 = p* - 1.5 u^2 - 1.5 u.a - tr(B) / 3,   K1 = 3 - 4.5 u^2 - tr(B),   v = 1.5 a - 2 B u
(cu = c_i.u, ca = c_i.a, cBc = c_i^T B c_i).  These tests take the oracle's collision (Eq. LBexp
with Eqs. eqts, noneqts and the forcing, built from Hermite tensors) of arbitrary pre-collision
populations and check, node by node:
  * the oracle's 27 post-collision populations equal the polynomial of (p*, u, a, B);
  * their moments give the set back: sum g = p*, sum g c = u + a / 2 and
    sum g c c = p* I / 3 + (2/9) (B + 4.5 u u + 4.5 sym(u a)), the import that lbm_set_state uses;
  * negating the components odd in x (u_x, a_x, B_xy, B_xz) maps direction (cx, cy, cz) to
    (-cx, cy, cz), the mirror the tiled kernel uses for one halo column.
"""
import numpy as np

import oracle

C = np.array([(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)], dtype=np.float64)
_N2 = (C * C).sum(1)
W = np.select([_N2 == 0, _N2 == 1, _N2 == 2, _N2 == 3], [8 / 27, 2 / 27, 1 / 54, 1 / 216])


def polynomial(ps, u, a, B):
    """g_i of the moment set, all 27 directions."""
    cu, ca, cv = C @ u, C @ a, None
    cBc = np.einsum("ia,ab,ib->i", C, B, C)
    trB = np.trace(B)
    K0 = ps - 1.5 * u @ u - 1.5 * u @ a - trB / 3
    K1 = 3 - 4.5 * u @ u - trB
    v = 1.5 * a - 2 * B @ u
    cv = C @ v
    return W * (K0 + 4.5 * cu * (cu + ca) + cBc + cu * (K1 + 4.5 * cu * cu + 3 * cBc) + cv)


def _collide(rng):
    """Arbitrary pre-collision populations (not in the Hermite span), an acceleration and omega."""
    pstar = rng.normal(scale=0.05)
    u = rng.normal(scale=0.05, size=3)
    f = oracle.equilibrium(pstar, u) + W * rng.normal(scale=2e-3, size=27)
    acc = rng.normal(scale=1e-3, size=3)
    omega = rng.uniform(0.3, 1.95)
    g, uu, A = oracle.collide_node(f, acc, omega)
    return f, acc, omega, g, uu, A


def test_post_collision_populations_are_the_moment_polynomial():
    rng = np.random.default_rng(2501)
    for _ in range(300):
        f, acc, omega, g, u, A = _collide(rng)
        B = 4.5 * (1 - omega) * A
        np.testing.assert_allclose(polynomial(f.sum(), u, acc, B), g, rtol=0, atol=1e-15)


def test_population_moments_give_the_set_back():
    rng = np.random.default_rng(2502)
    for _ in range(300):
        f, acc, omega, g, u, A = _collide(rng)
        B = 4.5 * (1 - omega) * A
        ps = g.sum()
        assert abs(ps - f.sum()) < 1e-15
        a = 2 * (C.T @ g - u)
        np.testing.assert_allclose(a, acc, rtol=0, atol=1e-15)
        Pi = np.einsum("i,ia,ib->ab", g, C, C)
        T = 4.5 * (Pi - ps / 3 * np.eye(3))
        B_back = T - 4.5 * np.outer(u, u) - 2.25 * (np.outer(u, a) + np.outer(a, u))
        np.testing.assert_allclose(B_back, B, rtol=0, atol=1e-14)


def test_import_is_the_hermite_projection_for_any_populations():
    """For populations outside the polynomial's span, expanding the imported set keeps p*, the
    momentum and the second moment of the input (what the projection preserves)."""
    rng = np.random.default_rng(2503)
    for _ in range(100):
        g = W * (0.1 + rng.normal(scale=0.01, size=27))
        u = rng.normal(scale=0.05, size=3)
        ps = g.sum()
        a = 2 * (C.T @ g - u)
        T = 4.5 * (np.einsum("i,ia,ib->ab", g, C, C) - ps / 3 * np.eye(3))
        B = T - 4.5 * np.outer(u, u) - 2.25 * (np.outer(u, a) + np.outer(a, u))
        h = polynomial(ps, u, a, B)
        assert abs(h.sum() - ps) < 1e-14
        np.testing.assert_allclose(C.T @ h, C.T @ g, rtol=0, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", h, C, C), np.einsum("i,ia,ib->ab", g, C, C),
                                   rtol=0, atol=1e-14)


def test_x_mirror_of_the_moments_mirrors_the_directions():
    rng = np.random.default_rng(2504)
    mirror = np.array([9 * (cz + 1) + 3 * (cy + 1) + (1 - cx) for cx, cy, cz in C.astype(int)])
    for _ in range(100):
        f, acc, omega, g, u, A = _collide(rng)
        B = 4.5 * (1 - omega) * A
        S = np.diag([-1.0, 1.0, 1.0])
        gm = polynomial(f.sum(), S @ u, S @ acc, S @ B @ S)
        np.testing.assert_allclose(gm, g[mirror], rtol=0, atol=1e-15)
