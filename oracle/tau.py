"""Stabilisation matrix tau of eq. (3D-tau), section 2.2.

tau = [ A_i G_ij A_j + C_I kappa^2 G_ij G_ij I ]^{-1/2}

computed as the paper describes after eq. (3D-tau): form the matrix under
the root, take its eigenpairs, apply lambda^{-1/2} to the eigenvalues and
multiply back with the eigenvectors.  The eigensolver is numpy's Hermitian
routine (a library primitive used as one step).  For the Navier-Stokes
operator kappa is the kinematic viscosity mu / rho (a reading: the paper
says the design is identical to eq. 3D-tau; App. B eq. 3D-taut is its
one-mode case).

Pinned by: tests/test_oracle_tau.py (tau M tau = I; Hermitian positive
definite; tau_{-m,-n} = conj(tau_{mn}); one-mode and mode-0-only limits equal
the scalar formula of eq. 3D-taut with omega_hat = 0; A = 0 gives the pure
diffusive limit; the 1D reduction equals eq. 1D-Stau and its eigenvalue
form eq. 1D-tauT).
"""
from __future__ import annotations

import numpy as np


def tau_argument(A: np.ndarray, G: np.ndarray, kappa: float, C_I: float) -> np.ndarray:
    """M = sum_ij G_ij A_i A_j + C_I kappa^2 (G:G) I.  A: [...,3,nm,nm], G: [...,3,3]."""
    nm = A.shape[-1]
    M = np.einsum("...ij,...imn,...jnk->...mk", G.astype(np.complex128), A, A)
    GG = np.einsum("...ij,...ij->...", G, G)
    M = M + (C_I * kappa * kappa * GG)[..., None, None] * np.eye(nm)
    return M


def inv_sqrt_hermitian(M: np.ndarray) -> np.ndarray:
    M = 0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))
    lam, V = np.linalg.eigh(M)
    if np.any(lam <= 0):
        raise FloatingPointError("tau argument is not positive definite")
    return np.einsum("...mk,...k,...nk->...mn", V, lam ** -0.5, np.conj(V))


def tau_matrix(A: np.ndarray, G: np.ndarray, kappa: float, C_I: float) -> np.ndarray:
    return inv_sqrt_hermitian(tau_argument(A, G, kappa, C_I))
