"""Pins for oracle.precond (the nodal block preconditioners).

The colour sweeps of the symmetric block Gauss-Seidel method are checked
against its closed form z = (D + U)^{-1} D (D + L)^{-1} x, formed with dense
triangular-by-blocks matrices and a library solve; block Jacobi against a
dense solve of the block diagonal.  The matrices are random, with a random
node coupling graph, a greedy colouring of it and random fixed unknowns.
"""
import numpy as np
import pytest

from oracle import precond as pc


def _random_system(seed, V=14, nb=4, p_edge=0.3, p_fixed=0.15):
    rng = np.random.default_rng(seed)
    adj = rng.random((V, V)) < p_edge
    adj = adj | adj.T
    np.fill_diagonal(adj, True)
    H = rng.standard_normal((V, nb, V, nb)) * adj[:, None, :, None]
    for A in range(V):   # diagonally dominant blocks: the sweeps are well defined
        H[A, :, A, :] += 4.0 * nb * np.eye(nb)
    fixed = rng.random((V, nb)) < p_fixed
    # greedy colouring of the coupling graph, in node order
    colour = -np.ones(V, dtype=int)
    for A in range(V):
        used = {colour[B] for B in range(V) if adj[A, B] and B != A and colour[B] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[A] = c
    x = rng.standard_normal((V, nb))
    x[fixed] = 0.0
    return H, fixed, colour, x


def _dense(D_inv, off):
    V, nb = D_inv.shape[:2]
    D = np.zeros((V * nb, V * nb))
    for A in range(V):
        D[A * nb:(A + 1) * nb, A * nb:(A + 1) * nb] = np.linalg.inv(D_inv[A])
    return D, off.reshape(V * nb, V * nb)


def _closed_form(D_inv, off, colour, x):
    V, nb = x.shape
    D, O = _dense(D_inv, off)
    below = (colour[:, None] > colour[None, :]).astype(float)   # colour(B) < colour(A)
    above = (colour[:, None] < colour[None, :]).astype(float)
    L = O * np.kron(below, np.ones((nb, nb)))
    U = O * np.kron(above, np.ones((nb, nb)))
    xv = x.ravel()
    z1 = np.linalg.solve(D + L, xv)
    return np.linalg.solve(D + U, D @ z1).reshape(V, nb)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gauss_seidel_sweeps_equal_the_closed_form(seed):
    H, fixed, colour, x = _random_system(seed)
    D_inv, off = pc.masked_blocks(H, fixed)
    assert pc.check_colouring(off, colour)
    assert colour.max() >= 2                      # several colours, so L and U are not empty
    z = pc.symmetric_block_gauss_seidel(D_inv, off, colour, x)
    ref = _closed_form(D_inv, off, colour, x)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.all(z[fixed] == 0.0)
    # one node per colour: the point-ordered block method, same closed form
    order = np.arange(len(colour))
    z_pt = pc.symmetric_block_gauss_seidel(D_inv, off, order, x)
    ref_pt = _closed_form(D_inv, off, order, x)
    assert np.linalg.norm(z_pt - ref_pt) <= 1e-12 * np.linalg.norm(ref_pt)
    # the colour order matters: reversing it gives a different (valid) result
    z_rev = pc.symmetric_block_gauss_seidel(D_inv, off, colour.max() - colour, x)
    assert np.linalg.norm(z_rev - z) > 1e-6 * np.linalg.norm(z)


def test_block_jacobi_is_a_solve_of_the_block_diagonal():
    H, fixed, colour, x = _random_system(3)
    D_inv, off = pc.masked_blocks(H, fixed)
    D, _ = _dense(D_inv, off)
    z = pc.block_jacobi(D_inv, x)
    assert np.allclose(z.ravel(), np.linalg.solve(D, x.ravel()), rtol=1e-12, atol=1e-14)
    # fixed unknowns: identity rows and columns in the blocks, none off them
    for A in range(x.shape[0]):
        Dm = np.linalg.inv(D_inv[A])
        f = fixed[A]
        assert np.allclose(Dm[np.ix_(f, f)], np.eye(f.sum()))
        assert np.all(Dm[np.ix_(f, ~f)] == 0.0) and np.all(Dm[np.ix_(~f, f)] == 0.0)
        assert np.all(off[A, f] == 0.0) and np.all(off[:, :, A, f] == 0.0)
    # no off-diagonal coupling: Gauss-Seidel reduces to block Jacobi
    z_gs = pc.symmetric_block_gauss_seidel(D_inv, np.zeros_like(off), colour, x)
    assert np.allclose(z_gs, z, rtol=1e-13, atol=1e-15)


def test_colouring_check_rejects_coupled_nodes_of_one_colour():
    H, fixed, colour, x = _random_system(4)
    D_inv, off = pc.masked_blocks(H, fixed)
    assert pc.check_colouring(off, colour)
    A, B = np.argwhere(np.abs(off).sum(axis=(1, 3)) > 0)[0]
    bad = colour.copy()
    bad[B] = bad[A]
    assert not pc.check_colouring(off, bad)
