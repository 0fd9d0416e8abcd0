"""Pins for the backflow stabilisation term of section 2.6 in the oracle."""
import numpy as np

from oracle import operator as op
from oracle.geometry import face_normals_areas
from workloads import cases, meshgen as mg


def _prob(mesh, N, beta=None, omega=0.7, rho=1.3, mu=0.05):
    dmask = cases.dirichlet_nodes(mesh, (mg.TAG_WALL, mg.TAG_INLET1))
    out = mesh.bfaces[mesh.btag == mg.TAG_OUTLET1]
    bf = [(out, beta)] if beta is not None else []
    return op.make_problem(mesh.xyz, mesh.tets, N, rho, mu, omega, dmask, 3.0, [], bf)


def _axial_state(mesh, N, coeffs):
    """u = (0, 0, w(t)) with w(t) = sum_n c_n e^{i n w t}, uniform in space."""
    y = np.zeros((mesh.n_nodes, 4, N, 2))
    for n, c in enumerate(coeffs[:N]):
        y[:, 2, n, 0] = np.real(c)
        y[:, 2, n, 1] = 0.0 if n == 0 else np.imag(c)
    return y


def test_no_backflow_leaves_the_residual_unchanged():
    # w(t) = 1 + 2*0.4 cos(wt) + 2*0.1 cos(2wt) > 0: A_n is the Toeplitz section of a
    # positive symbol, hence positive semi-definite, and |A_n|_- = 0 (section 2.6 remark 2)
    mesh = mg.pipe(nc=2, nr=1, nz=3, seed=2)
    N = 3
    y = _axial_state(mesh, N, [1.0, 0.4, 0.1]) + 0.01 * cases.random_state(mesh, N, seed=1)
    r0 = op.residual(_prob(mesh, N), y)
    r1 = op.residual(_prob(mesh, N, beta=1.0), y)
    np.testing.assert_allclose(r1, r0, atol=1e-13 * np.abs(r0).max())


def test_single_mode_reduces_to_the_scalar_time_formulation_term():
    # N = 1: |A_n|_- = min(u.n, 0); the term is -int N_A (rho/2) beta min(u.n, 0) u_i
    mesh = mg.pipe(nc=2, nr=1, nz=3, seed=3)
    prob0, prob1 = _prob(mesh, 1), _prob(mesh, 1, beta=0.7)
    y = cases.random_state(mesh, 1, seed=4)
    y[:, 2] -= 0.8                                   # mostly inflow through the outlet
    diff = op.residual(prob1, y) - op.residual(prob0, y)
    faces = mesh.bfaces[mesh.btag == mg.TAG_OUTLET1]
    n, area = face_normals_areas(mesh.xyz, faces)
    ref = np.zeros((mesh.n_nodes, 3))
    bary = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
    for f in range(faces.shape[0]):
        u = y[faces[f], 0:3, 0, 0]                   # [3 vertices, 3]
        for g in range(3):
            ug = bary[g] @ u
            un = ug @ n[f]
            for b in range(3):
                ref[faces[f, b]] += -(area[f] / 3) * bary[g, b] * 0.5 * prob1.rho * 0.7 * min(un, 0.0) * ug
    ref[prob1.dmask] = 0.0
    assert np.abs(ref).max() > 1e-3
    np.testing.assert_allclose(diff[:, 0:3, 0, 0], ref, atol=1e-13 * np.abs(ref).max())
    assert np.abs(diff[:, 3]).max() == 0.0


def test_backflow_term_only_adds_dissipation():
    # u^H (term) = -(rho/2) beta int u^H |A_n|_- u >= 0 for any field (|A_n|_- <= 0)
    mesh = mg.pipe(nc=2, nr=1, nz=3, seed=5)
    N = 4
    prob0, prob1 = _prob(mesh, N), _prob(mesh, N, beta=1.0)
    y = cases.random_state(mesh, N, seed=6)
    y[:, 2, 0, 0] -= 0.5
    lin = op.linearize(prob1, y)
    assert any(np.abs(B).max() > 1e-3 for B in lin.Bneg)
    for B in lin.Bneg:
        assert np.linalg.eigvalsh(B).max() < 1e-12
    dc = op.residual(prob1, y, return_complex=True) - op.residual(prob0, y, return_complex=True)
    from oracle.spectral import to_complex
    U = to_complex(y, N)
    energy = np.real(np.sum(np.conj(U[:, 0:3]) * dc[:, 0:3]))
    assert energy > 0
