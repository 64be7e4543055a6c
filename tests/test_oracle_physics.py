"""Whole-step pins of the oracle against closed forms of the continuum problem.

Each case is small (1D or 2D boxes) so the CPU suite stays fast; every tolerance is either the
measured discretisation error of the scheme with margin, or a convergence-order statement (the
error falls by ~4x when the interface width and the grid are doubled).

  * conservation: sum(phi) and sum(p*) are invariants of one step (every Allen-Cahn term is a
    discrete divergence or Laplacian; streaming permutes populations; collision keeps p*);
  * planar interface: the tanh profile (reading R9) is the equilibrium of the Allen-Cahn
    update, to second order in 1/W;
  * Laplace law: a 2D droplet has p_in - p_out = sigma/R (sphere: 2 sigma/R);
  * two-layer Poiseuille with walls: steady d/dz(mu du/dz) = -G with no slip; this pins the
    viscous-correction force F^nu (Eq. visc_corr) and the viscosity interpolation;
  * hydrostatics: dp/dz = (rho - rho_ref) g; this pins F^p (Eq. press_corr) and p = p* rho cs^2;
  * Taylor-Green decay exp(-2 nu k^2 t) in the single-phase limit;
  * uniform translation of a droplet (Galilean check of the coupled step).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_00846_b300 import inputs


def _zero_u(P):
    return np.zeros((3,) + P.shape)


@pytest.mark.parametrize("wall", [0, 1])
def test_conservation_of_phi_and_pstar(wall):
    L = 14
    P = oracle.Params(L, L - 1, L + 2, wall_z=wall, rho_l=1.0, rho_g=0.01, mu_l=0.05, mu_g=0.005,
                      sigma=0.01, gravity=(0.0, 0.0, -1e-5) if wall else (0.0, 0.0, 0.0))
    phi = inputs.sphere_phi(P.nx, P.ny, P.nz, (6.3, 5.8, 7.7), 4.0, 4.0,
                            periodic=(True, True, not wall))
    u = inputs.fourier_velocity(P.nx, P.ny, P.nz, amplitude=0.02, seed=3)
    if wall:
        u = inputs.wall_damp(u, P.nz)
    s0 = oracle.init(P, phi, u, pstar0=0.01 * np.sin(np.arange(P.n)).reshape(P.shape))
    sphi0, sps0 = s0.phi.sum(), oracle.pstar(s0).sum()
    s = s0
    for _ in range(6):
        s = oracle.run(P, s, 10)
        assert abs(s.phi.sum() - sphi0) < 1e-12 * sphi0
        assert abs(oracle.pstar(s).sum() - sps0) < 1e-12
    assert np.isfinite(s.g).all()


@pytest.mark.parametrize("W", [4.0, 8.0])
def test_planar_interface_is_stationary(W):
    """1D slab, u = 0: after relaxation the profile stays within O(1/W^2) of the tanh."""
    nz = int(16 * W)
    P = oracle.Params(1, 1, nz, sigma=0.01, width=W)
    phi = inputs.slab_phi(1, 1, nz, nz / 4 - 0.5, 3 * nz / 4 - 0.5, W)
    s = oracle.run(P, oracle.init(P, phi, _zero_u(P)), 3000)
    dev = np.abs(s.phi - phi).max()
    # measured: 5.3e-3 at W = 4, 1.5e-3 at W = 8 (second order)
    assert dev < {4.0: 7e-3, 8.0: 2e-3}[W]
    assert abs(s.phi.sum() - phi.sum()) < 1e-12 * phi.sum()


def _laplace_2d(R, L=48, sigma=0.01, steps=2000):
    P = oracle.Params(L, L, 1, sigma=sigma)
    c = (L - 1) / 2.0
    phi = inputs.cylinder_phi(L, L, 1, (c, c), R, 4.0)
    s = oracle.run(P, oracle.init(P, phi, _zero_u(P)), steps)
    o = oracle.observables(P, s)
    Reff = math.sqrt(s.phi.sum() / math.pi)
    return o["p_liq"] - o["p_gas"], Reff, o


def test_laplace_law_2d():
    sigma = 0.01
    dps, inv_r = [], []
    for R in (8.0, 10.0, 12.0):
        dp, Reff, o = _laplace_2d(R, sigma=sigma)
        # measured ratios 0.997 / 0.984 / 0.978
        assert abs(dp / (sigma / Reff) - 1.0) < 0.03, (R, dp, sigma / Reff)
        assert o["umax"] < 1e-4            # spurious currents stay small
        dps.append(dp)
        inv_r.append(1.0 / Reff)
    slope = np.polyfit(inv_r, dps, 1)[0]
    assert abs(slope / sigma - 1.0) < 0.05


def _diffuse_poiseuille(nz, zi, W, G, mu_l, mu_g):
    """Exact steady solution of d/dz(mu(z) du/dz) = -G, u(-1/2) = u(nz-1/2) = 0, with mu(z)
    interpolated linearly in the tanh phase field (quadrature on a fine grid)."""
    zf = np.linspace(-0.5, nz - 0.5, 400001)
    ph = 0.5 + 0.5 * np.tanh(2 * (zi - zf) / W)
    mu = mu_g + ph * (mu_l - mu_g)

    def integ(c1):
        d = (-G * zf + c1) / mu
        return np.concatenate([[0.0], np.cumsum(0.5 * (d[1:] + d[:-1]) * np.diff(zf))])

    i0 = integ(0.0)
    i1 = integ(1.0) - i0
    c1 = -i0[-1] / i1[-1]
    return np.interp(np.arange(nz), zf, i0 + c1 * i1)


def _poiseuille_error(nz, W, G=1e-6):
    mu_l, mu_g = 1.0 / 6.0, 1.0 / 60.0        # viscosity ratio 10, density ratio 10, nu = 1/6
    P = oracle.Params(1, 1, nz, wall_z=1, rho_l=1.0, rho_g=0.1, mu_l=mu_l, mu_g=mu_g,
                      sigma=0.01, width=W, body=(G, 0.0, 0.0))
    zi = (nz - 1) / 2.0
    phi = inputs.layer_phi(1, 1, nz, zi, W)
    steps = int(10 * nz * nz / (math.pi ** 2 / 6.0))     # ~10 viscous times
    s = oracle.run(P, oracle.init(P, phi, _zero_u(P)), steps)
    u = s.u[0, :, 0, 0]
    ue = _diffuse_poiseuille(nz, zi, W, G, mu_l, mu_g)
    assert np.abs(s.u[1:]).max() < 1e-8
    return math.sqrt(((u - ue) ** 2).sum() / (ue ** 2).sum())


def test_two_layer_poiseuille():
    e1 = _poiseuille_error(32, 4.0)
    e2 = _poiseuille_error(64, 8.0)
    # measured 8.5e-3 and 2.4e-3: second-order convergence towards the exact profile
    assert e1 < 0.015
    assert e2 < 0.004
    assert e1 / e2 > 3.0


def _hydrostatic_ratio(W, nz=48, g=1e-5):
    P = oracle.Params(1, 1, nz, wall_z=1, rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.0,
                      width=W, gravity=(0.0, 0.0, -g), rho_ref=1.0)
    phi = inputs.layer_phi(1, 1, nz, (nz - 1) / 2.0, W)
    s = oracle.run(P, oracle.init(P, phi, _zero_u(P)), 12000)
    p = oracle.pressure(P, s)[:, 0, 0]
    rho = oracle.density(P, s.phi)[:, 0, 0]
    # dp/dz = (rho - rho_ref) g_z = (1 - rho) g, trapezoidal integral over the nodes
    head = (0.5 * ((1 - rho[1:]) + (1 - rho[:-1]))).sum() * g
    assert np.abs(s.u).max() < 1e-5
    return (p[-1] - p[0]) / head


def test_hydrostatic_balance():
    r4 = _hydrostatic_ratio(4.0)
    r8 = _hydrostatic_ratio(8.0)
    # measured 0.972 and 0.994: the error sits inside the diffuse interface, second order in 1/W
    assert abs(r4 - 1) < 0.04
    assert abs(r8 - 1) < 0.01
    assert abs(r4 - 1) / abs(r8 - 1) > 3.0


def test_taylor_green_decay():
    L, nu, U, steps = 32, 0.05, 0.01, 300
    P = oracle.Params(L, L, 1, rho_l=1.0, rho_g=1.0, mu_l=nu, mu_g=nu, sigma=0.0)
    k = 2 * math.pi / L
    _, y, x = np.meshgrid(np.arange(1.0), np.arange(float(L)), np.arange(float(L)), indexing="ij")
    u = np.zeros((3,) + P.shape)
    u[0] = U * np.sin(k * x) * np.cos(k * y)
    u[1] = -U * np.cos(k * x) * np.sin(k * y)
    p = -(U * U / 4) * (np.cos(2 * k * x) + np.cos(2 * k * y))
    s = oracle.run(P, oracle.init(P, np.ones(P.shape), u, pstar0=3.0 * p), steps)
    amp = (s.u[0] * u[0]).sum() / (u[0] ** 2).sum()
    rate = -math.log(amp) / steps
    # measured relative rate error 4.7e-3 at L = 32
    assert abs(rate / (2 * nu * k * k) - 1) < 0.01


def test_droplet_translation():
    """A droplet in a uniform stream is carried at the stream velocity."""
    L, U, steps = 24, 0.02, 250
    P = oracle.Params(L, L, L, rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.005)
    phi = inputs.sphere_phi(L, L, L, (8.0, 11.5, 11.5), 5.0, 4.0)
    u = np.zeros((3,) + P.shape)
    u[0] = U
    s0 = oracle.init(P, phi, u)
    s = oracle.run(P, s0, steps)
    o0, o = oracle.observables(P, s0), oracle.observables(P, s)
    dx = o["centroid_liq"][0] - o0["centroid_liq"][0]
    assert abs(dx / (U * steps) - 1) < 0.02
    assert abs(o["centroid_liq"][1] - o0["centroid_liq"][1]) < 1e-6
    assert abs(o["vel_liq"][0] / U - 1) < 0.02


def test_sharpening_weight_vanishes_outside_unit_interval():
    """Reading R15: outside [0, 1] the sharpening weight phi (1 - phi) is zero, so at rest the
    Allen-Cahn update there reduces to FTCS diffusion phi + D lap(phi); inside (0, 1) it is not."""
    rng = np.random.default_rng(17)
    P = oracle.Params(8, 7, 6, mobility=0.1)
    above = 1.0 + 1e-3 * rng.random(P.shape)
    zero_u = np.zeros((3,) + P.shape)
    np.testing.assert_allclose(oracle.ac_update(P, above, zero_u), above + 0.1 * oracle.lap(P, above), atol=1e-15)
    below = -1e-3 * rng.random(P.shape)
    np.testing.assert_allclose(oracle.ac_update(P, below, zero_u), below + 0.1 * oracle.lap(P, below), atol=1e-15)
    inside = 0.5 + 0.1 * rng.random(P.shape)
    assert np.abs(oracle.ac_update(P, inside, zero_u) - (inside + 0.1 * oracle.lap(P, inside))).max() > 1e-4


def _grad27(psi):
    """3 sum_i w_i c_i psi(x + c_i) on a periodic box, written out with np.roll (psi[z, y, x])."""
    g = np.zeros((3,) + psi.shape)
    w1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    for cz in (-1, 0, 1):
        for cy in (-1, 0, 1):
            for cx in (-1, 0, 1):
                w = w1[cx] * w1[cy] * w1[cz]
                s = np.roll(psi, shift=(-cz, -cy, -cx), axis=(0, 1, 2))
                g[0] += 3 * w * cx * s
                g[1] += 3 * w * cy * s
                g[2] += 3 * w * cz * s
    return g


def test_literal_advection_form():
    """Reading R4 and its alternative.  The literal update phi - ubar . G[phi] equals the flux form
    phi - G . (ubar phi) when ubar is uniform (G is linear), and otherwise changes sum phi by
    exactly -sum ubar . G[phi] per step (every other term telescopes)."""
    L = 12
    base = dict(rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.01)
    phi = inputs.sphere_phi(L, L, L, (5.3, 6.1, 5.7), 3.5, 4.0, periodic=(True, True, True))
    P0, P1 = oracle.Params(L, L, L, advect=0, **base), oracle.Params(L, L, L, advect=1, **base)

    uni = np.zeros((3,) + P0.shape)
    uni[0], uni[1], uni[2] = 0.013, -0.007, 0.021
    a, b = oracle.ac_update(P0, phi, uni), oracle.ac_update(P1, phi, uni)
    assert np.abs(a - b).max() < 1e-15

    u = inputs.fourier_velocity(L, L, L, amplitude=0.02, seed=11)   # not divergence-free
    a, b = oracle.ac_update(P0, phi, u), oracle.ac_update(P1, phi, u)
    assert abs(a.sum() - phi.sum()) < 1e-12 * phi.sum()
    drift = -(u * _grad27(phi)).sum()
    assert abs(drift) > 1e-4
    assert abs((b.sum() - phi.sum()) - drift) < 1e-12 * phi.sum()


def test_literal_sharpening_weight_differs_only_where_phi_leaves_the_unit_interval():
    """Reading R15 against the printed weight phi (1 - phi) (Params.literal_weight = 1).  On a
    field inside [0, 1] the two updates are the same bits.  With planted overshoots the difference
    of one update is exactly -kappa_AC div(min(phi (1 - phi), 0) n) (the term R15 drops), the
    printed weight's sharpening flux at the overshoots, and both forms conserve sum phi."""
    L = 10
    base = dict(rho_l=1.0, rho_g=0.1, mu_l=0.1, mu_g=0.01, sigma=0.01, mobility=0.1, width=4.0)
    P0, P1 = oracle.Params(L, L, L, **base), oracle.Params(L, L, L, literal_weight=1, **base)
    phi = inputs.sphere_phi(L, L, L, (4.6, 5.2, 4.9), 3.0, 4.0, periodic=(True, True, True))
    u = inputs.fourier_velocity(L, L, L, amplitude=0.01, seed=3)
    assert phi.min() >= 0.0 and phi.max() <= 1.0
    assert np.array_equal(oracle.ac_update(P0, phi, u), oracle.ac_update(P1, phi, u))
    rng = np.random.default_rng(5)
    over = phi.copy()
    bulk = np.abs(phi - 0.5) > 0.3              # plant overshoots in both bulk phases
    over[bulk] += np.sign(phi[bulk] - 0.5) * 0.02 * rng.random(int(bulk.sum()))
    over[bulk] = np.where(phi[bulk] > 0.5, np.maximum(over[bulk], 1.0 + 1e-3 * rng.random(int(bulk.sum()))),
                          np.minimum(over[bulk], -1e-3 * rng.random(int(bulk.sum()))))
    assert over.max() > 1.0 and over.min() < 0.0
    a, b = oracle.ac_update(P0, over, u), oracle.ac_update(P1, over, u)
    g = oracle.grad(P0, over)
    n = g / np.maximum(np.sqrt((g ** 2).sum(axis=0)), 1e-12)
    dropped = np.minimum(over * (1.0 - over), 0.0)
    kac = 4.0 * P0.mobility / P0.width
    expect = -kac * oracle.div(P0, dropped[None] * n)
    assert np.abs(b - a).max() > 1e-6
    np.testing.assert_allclose(b - a, expect, atol=1e-15)
    assert abs(a.sum() - over.sum()) < 1e-12 * over.sum() and abs(b.sum() - over.sum()) < 1e-12 * over.sum()
