"""Closed-form time-periodic flow in a straight rigid pipe (Womersley 1955).

The paper cites laminar pipe flow as a case with a unique time-periodic
solution (section 2.4).  Fully developed flow has u.grad u = 0, so the
closed form is an exact Navier-Stokes solution and the time-spectral modes
decouple:

  mode 0 (Poiseuille):  w_0(r) = 2 U_0 (1 - r^2/R^2),  -dp_0/dz = 8 mu U_0 / R^2
  mode n >= 1:          w_n(r) = (G_n / (i rho n omega)) [1 - J0(L r/R) / J0(L)]
                        L = i^{3/2} alpha_n, alpha_n = R sqrt(n omega / nu)
                        U_n = (G_n / (i rho n omega)) [1 - 2 J1(L) / (L J0(L))]
                        p_n(z) = G_n (z_out - z)

with U_n the mean velocity of mode n.  J0 and J1 are summed from their
power series here (own implementation, no library Bessel routine), which
converges to round-off for |z| <~ 20 (kept alpha_n <= 15 in tests).

Pinned by: tests/test_oracle_womersley.py (series against scipy's complex
Bessel functions and the Kelvin-function values ber/bei; the alpha -> 0
limit equals Poiseuille; the profile satisfies the mode ODE
i rho n omega w = G + mu (w'' + w'/r) by finite differences and w(R) = 0).
Parity unpinned for alpha_n > 15.
"""
from __future__ import annotations

import math

import numpy as np


def bessel_j(nu: int, z, terms: int = 80):
    """J_nu(z) for integer nu >= 0 by its power series."""
    z = np.asarray(z, dtype=np.complex128)
    half = z / 2.0
    term = half ** nu / math.factorial(nu)
    total = term.copy()
    h2 = half * half
    for k in range(1, terms):
        term = term * (-h2) / (k * (k + nu))
        total = total + term
    return total


def mode_profile(r, R, Un, n, omega, nu):
    if n == 0:
        return 2.0 * Un * (1.0 - (np.asarray(r) / R) ** 2)
    alpha = R * math.sqrt(n * omega / nu)
    L = (1j) ** 1.5 * alpha
    j0 = bessel_j(0, L)
    shape = 1.0 - bessel_j(0, L * np.asarray(r) / R) / j0
    mean_shape = 1.0 - 2.0 * bessel_j(1, L) / (L * j0)
    return Un * shape / mean_shape


def pressure_gradient(R, Un, n, rho, mu, omega):
    """G_n = -dp_n/dz."""
    if n == 0:
        return 8.0 * mu * Un / R ** 2
    nu = mu / rho
    alpha = R * math.sqrt(n * omega / nu)
    L = (1j) ** 1.5 * alpha
    mean_shape = 1.0 - 2.0 * bessel_j(1, L) / (L * bessel_j(0, L))
    return Un * 1j * rho * n * omega / mean_shape


def pipe_solution(xyz, R, L, U, rho, mu, omega):
    """Storage-layout field [V,4,N,2] of the closed form (axis z, outlet at z = L)."""
    N = len(U)
    V = xyz.shape[0]
    y = np.zeros((V, 4, N, 2))
    r = np.hypot(xyz[:, 0], xyz[:, 1])
    for n in range(N):
        w = mode_profile(r, R, U[n], n, omega, mu / rho)
        p = pressure_gradient(R, U[n], n, rho, mu, omega) * (L - xyz[:, 2])
        y[:, 2, n, 0], y[:, 2, n, 1] = np.real(w), np.imag(w)
        y[:, 3, n, 0], y[:, 3, n, 1] = np.real(p), np.imag(p)
    y[:, :, 0, 1] = 0.0
    return y
