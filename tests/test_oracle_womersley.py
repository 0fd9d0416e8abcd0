"""Pins for oracle.womersley (own Bessel series) and the closed-form flow."""
import math

import numpy as np
import pytest

from oracle import womersley as wo


def test_bessel_series_against_library_and_kelvin_values():
    scipy_special = pytest.importorskip("scipy.special")
    for alpha in (0.3, 2.5, 7.0, 15.0):
        z = (1j) ** 1.5 * alpha * np.linspace(0, 1, 9)
        for nu in (0, 1):
            ref = scipy_special.jv(nu, z)
            np.testing.assert_allclose(wo.bessel_j(nu, z), ref, rtol=1e-11, atol=1e-14)
    # Kelvin functions ber(x) + i bei(x) = J0(x e^{3 pi i / 4}); ber(1), bei(1) to 9 digits
    v = wo.bessel_j(0, (1j) ** 1.5 * 1.0)
    assert abs(v.real - 0.984381781) < 2e-9 and abs(v.imag - 0.249566040) < 2e-9


def test_small_alpha_tends_to_poiseuille_and_wall_is_no_slip():
    r = np.linspace(0, 1, 11)
    w = wo.mode_profile(r, 1.0, 0.7, 1, omega=1e-8, nu=1.0)
    np.testing.assert_allclose(w, 2 * 0.7 * (1 - r ** 2), rtol=1e-6, atol=1e-9)
    for alpha_case in (1.0, 9.0):
        w = wo.mode_profile(np.array([1.0]), 1.0, 0.3 + 0.2j, 2, omega=alpha_case ** 2 / 2, nu=1.0)
        assert abs(w[0]) < 1e-12


def test_profile_satisfies_mode_equation_and_mean_velocity():
    R, rho, mu, omega, n = 1.3, 1.1, 0.05, 0.8, 2
    Un = 0.4 - 0.25j
    G = wo.pressure_gradient(R, Un, n, rho, mu, omega)
    r = np.linspace(0.2, 1.1, 7)
    h = 1e-4
    w = wo.mode_profile(r, R, Un, n, omega, mu / rho)
    wp = wo.mode_profile(r + h, R, Un, n, omega, mu / rho)
    wm = wo.mode_profile(r - h, R, Un, n, omega, mu / rho)
    lap = (wp - 2 * w + wm) / h ** 2 + (wp - wm) / (2 * h) / r
    np.testing.assert_allclose(1j * rho * n * omega * w, G + mu * lap, rtol=1e-5, atol=1e-7)
    # mean over the cross-section equals U_n
    rr = np.linspace(0, R, 4001)
    ww = wo.mode_profile(rr, R, Un, n, omega, mu / rho)
    mean = np.trapezoid(2 * np.pi * rr * ww, rr) / (math.pi * R * R)
    np.testing.assert_allclose(mean, Un, rtol=1e-6)
