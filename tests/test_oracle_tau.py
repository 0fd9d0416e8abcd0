"""Pins for oracle.tau: eq. (3D-tau) and its special cases."""
import numpy as np

from oracle.spectral import conv_matrix, to_complex
from oracle.tau import tau_argument, tau_matrix


def _conj_sym(rng, N, scale=1.0):
    y = scale * rng.standard_normal((N, 2))
    y[0, 1] = 0.0
    return to_complex(y, N)


def _spd3(rng):
    B = rng.standard_normal((3, 3))
    return B @ B.T + 0.5 * np.eye(3)


def test_tau_is_inverse_square_root_hermitian_pd_and_symmetric_in_modes():
    rng = np.random.default_rng(0)
    for N in (1, 2, 4, 7):
        A = np.stack([conv_matrix(_conj_sym(rng, N)) for _ in range(3)])
        G = _spd3(rng)
        M = tau_argument(A, G, kappa=0.03, C_I=3.0)
        tau = tau_matrix(A, G, kappa=0.03, C_I=3.0)
        nm = 2 * N - 1
        np.testing.assert_allclose(tau @ M @ tau, np.eye(nm), atol=1e-11)
        np.testing.assert_allclose(tau, tau.conj().T, atol=1e-13)
        assert np.linalg.eigvalsh(tau).min() > 0
        # tau_{-m,-n} = conj(tau_{m,n}) (section 2.1 remark 5)
        np.testing.assert_allclose(tau[::-1, ::-1], tau.conj(), atol=1e-12)


def test_mode0_only_velocity_gives_scalar_time_formulation_tau():
    # A_i = u_i I  ->  tau = [u.G.u + C_I k^2 G:G]^{-1/2} I  (eq. 3D-taut, omega_hat = 0)
    rng = np.random.default_rng(1)
    N, kappa, C_I = 4, 0.02, 3.0
    u = rng.standard_normal(3)
    G = _spd3(rng)
    A = np.stack([u[i] * np.eye(2 * N - 1) for i in range(3)]).astype(complex)
    tau = tau_matrix(A, G, kappa, C_I)
    scalar = (u @ G @ u + C_I * kappa ** 2 * np.sum(G * G)) ** -0.5
    np.testing.assert_allclose(tau, scalar * np.eye(2 * N - 1), atol=1e-13)
    tau1 = tau_matrix(np.array([[[u[i]]] for i in range(3)], complex), G, kappa, C_I)
    np.testing.assert_allclose(tau1[0, 0], scalar, rtol=1e-13)


def test_zero_velocity_gives_diffusive_limit():
    rng = np.random.default_rng(2)
    G = _spd3(rng)
    A = np.zeros((3, 5, 5), complex)
    tau = tau_matrix(A, G, 0.04, 3.0)
    np.testing.assert_allclose(tau, (3.0 * 0.04 ** 2 * np.sum(G * G)) ** -0.5 * np.eye(5), rtol=1e-13)


def test_one_dimensional_reduction_matches_1d_formulas():
    # parent element of size 2: dxi/dx = 2/h, coefficient 9 -> eq. (1D-Stau)
    h, kappa, u = 0.3, 0.05, 1.7
    G = np.diag([(2 / h) ** 2, 0.0, 0.0])
    A = np.zeros((3, 1, 1), complex)
    A[0, 0, 0] = u
    tau = tau_matrix(A, G, kappa, C_I=9.0)
    ref = ((2 * u / h) ** 2 + (12 * kappa / h ** 2) ** 2) ** -0.5
    np.testing.assert_allclose(tau[0, 0].real, ref, rtol=1e-13)
    # unsteady: eigenvalues of tau from those of A via eq. (1D-tauT)
    rng = np.random.default_rng(3)
    N = 5
    A1 = conv_matrix(_conj_sym(rng, N))
    A = np.stack([A1, 0 * A1, 0 * A1])
    tau = tau_matrix(A, G, kappa, C_I=9.0)
    lam = np.linalg.eigvalsh(A1)
    ref = np.sort(((2 * lam / h) ** 2 + (12 * kappa / h ** 2) ** 2) ** -0.5)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(tau)), ref, rtol=1e-12)
