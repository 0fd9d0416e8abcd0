"""Nodal block preconditioners of the GMRES solve (test infrastructure only).

The paper's linear solver is GMRES on the tangent of eq. (K_mat) (section
2.4); a preconditioner changes the Krylov path only, not the converged
field.  These are the two block forms the library offers, written out on a
matrix given as nodal blocks H[A, :, B, :] (node A's unknowns, node B's):

* block Jacobi: z_A = D_A^{-1} x_A with D_A = H[A, :, A, :];
* symmetric block Gauss-Seidel over a node colouring in which no two nodes
  of one colour are coupled: a forward sweep over the colours in increasing
  order from z = 0, then a backward sweep in decreasing order, each setting
  z_A = D_A^{-1} (x_A - sum_{B != A} H[A, :, B, :] z_B) for every node of the
  colour with the z of the colours already visited.  With L and U the parts
  of H below and above the block diagonal in colour order, the result is
  z = (D + U)^{-1} D (D + L)^{-1} x.

Fixed unknowns (Dirichlet velocity, Im of mode 0) are handled as the
library does: identity rows and columns in D_A, no coupling in the
off-diagonal blocks, zero entries of x.

Pinned by: tests/test_oracle_precond.py (the sweeps against the closed form
(D + U)^{-1} D (D + L)^{-1} with dense solves; block Jacobi against a dense
solve of the block-diagonal part; a single colour per node reduces Gauss-
Seidel to the plain point-ordered method; the colouring condition is
checked).
"""
from __future__ import annotations

import numpy as np


def masked_blocks(H: np.ndarray, fixed: np.ndarray):
    """(D_inv [V, nb, nb], off [V, nb, V, nb]) of H [V, nb, V, nb] with the
    fixed unknowns (bool [V, nb]) taken out: identity rows and columns in
    the diagonal blocks, zero rows and columns off the diagonal."""
    V, nb = fixed.shape
    D_inv = np.empty((V, nb, nb))
    off = H.copy()
    for A in range(V):
        D = H[A, :, A, :].copy()
        D[fixed[A], :] = 0.0
        D[:, fixed[A]] = 0.0
        D[fixed[A], fixed[A]] = 1.0
        D_inv[A] = np.linalg.inv(D)
        off[A, fixed[A], :, :] = 0.0
        off[:, :, A, fixed[A]] = 0.0
        off[A, :, A, :] = 0.0
    return D_inv, off


def block_jacobi(D_inv: np.ndarray, x: np.ndarray) -> np.ndarray:
    """z_A = D_A^{-1} x_A; x, z: [V, nb]."""
    return np.einsum("aij,aj->ai", D_inv, x)


def check_colouring(off: np.ndarray, colour: np.ndarray) -> bool:
    """No two distinct nodes of one colour are coupled by an off-diagonal block."""
    coupled = np.abs(off).sum(axis=(1, 3)) > 0
    same = colour[:, None] == colour[None, :]
    np.fill_diagonal(same, False)
    return not np.any(coupled & same)


def symmetric_block_gauss_seidel(D_inv: np.ndarray, off: np.ndarray, colour: np.ndarray,
                                 x: np.ndarray) -> np.ndarray:
    """Forward then backward colour sweeps from z = 0 (see the module text)."""
    n_col = int(colour.max()) + 1
    z = np.zeros_like(x)
    for order in (range(n_col), range(n_col - 1, -1, -1)):
        for c in order:
            nodes = np.nonzero(colour == c)[0]
            t = x[nodes] - np.einsum("aibj,bj->ai", off[nodes], z)
            z[nodes] = np.einsum("aij,aj->ai", D_inv[nodes], t)
    return z
