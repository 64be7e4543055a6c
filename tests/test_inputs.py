"""Pins of the seeded input generators and the dimensionless-group helpers."""
import math
import os

import numpy as np

from paper_2501_00846_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_rising_bubble_parameters_match_hand_derivation():
    ref = _golden("rising_bubble_params.txt")
    wl = inputs.rising_bubble()
    p = inputs.rising_bubble_params(sqrt_gR=0.02)
    assert math.isclose(-wl.gravity[2], ref["g"], rel_tol=1e-12)
    assert math.isclose(wl.sigma, ref["sigma"], rel_tol=1e-12)
    assert math.isclose(p["Ga"], ref["Ga"], rel_tol=1e-5)
    assert math.isclose(p["nu_l"], ref["nu_l"], rel_tol=1e-5)
    assert math.isclose(3 * wl.mu_l / wl.rho_l + 0.5, ref["tau_l"], rel_tol=1e-5)
    assert math.isclose(wl.mu_g, ref["mu_g"], rel_tol=1e-5)
    assert math.isclose(wl.rho_g, ref["rho_g"], rel_tol=1e-12)
    assert math.isclose(3 * wl.mu_g / wl.rho_g + 0.5, ref["tau_g"], rel_tol=1e-5)
    # Eo and Mo recovered from the parameters
    g = -wl.gravity[2]
    assert math.isclose(wl.rho_l * g * wl.radius ** 2 / wl.sigma, 10.0, rel_tol=1e-12)
    assert math.isclose(g * wl.mu_l ** 4 / (wl.rho_l * wl.sigma ** 3), 1e-4, rel_tol=1e-9)


def test_fourier_velocity_is_seeded_and_scaled():
    a = inputs.fourier_velocity(16, 12, 10, amplitude=0.01, seed=1234)
    b = inputs.fourier_velocity(16, 12, 10, amplitude=0.01, seed=1234)
    c = inputs.fourier_velocity(16, 12, 10, amplitude=0.01, seed=1235)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert math.isclose(np.sqrt((a ** 2).sum(0)).max(), 0.01, rel_tol=1e-12)


def test_sphere_profile():
    phi = inputs.sphere_phi(32, 32, 32, (15.5, 15.5, 15.5), 8.0, 4.0)
    assert phi.min() > 0 and phi.max() < 1
    assert phi[16, 16, 16] > 0.999 and phi[0, 0, 0] < 1e-3
    bub = inputs.sphere_phi(32, 32, 32, (15.5, 15.5, 15.5), 8.0, 4.0, inside=0.0)
    np.testing.assert_allclose(bub, 1 - phi)


def test_droplet_ensemble_draws():
    """The 256-box ensemble: seeded, sizes and properties inside the stated ranges, equal
    kinematic viscosity, and identical for the same seed."""
    a = inputs.droplet_ensemble()
    b = inputs.droplet_ensemble()
    assert len(a) == 256
    for wa, wb in zip(a, b):
        assert wa.params() == wb.params() and wa.radius == wb.radius and wa.noise == wb.noise
    L = np.array([w.nx for w in a])
    assert L.min() >= 32 and L.max() <= 96 and len(set(L)) > 30
    for w in a:
        assert w.nx == w.ny == w.nz and w.wall_z == 0
        assert 6.0 <= w.radius <= w.nx / 4.0
        assert 0.001 <= w.sigma <= 0.02
        assert 10.0 <= w.rho_l / w.rho_g <= 1000.0
        assert abs(w.mu_l / w.rho_l - w.mu_g / w.rho_g) < 1e-12
        assert 0.0 <= w.noise <= 0.02
    ratios = np.log10([w.rho_l / w.rho_g for w in a])
    assert abs(ratios.mean() - 2.0) < 0.15          # log-uniform over [1, 3] decades
    assert inputs.droplet_ensemble(seed=5)[0].params() != a[0].params()
