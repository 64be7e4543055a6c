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
