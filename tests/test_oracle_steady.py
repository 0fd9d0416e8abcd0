"""Pins for oracle.steady: the steady SUPG/PSPG residual of App. B eq. (NSt-weak).

``steady_residual`` pins the time-spectral residual's mode-0 limit, so it
needs pins of its own that do not share its code.  Each case below has a
closed form per element, assembled here with geometry computed another way
(barycentric gradients from inverting the 4x4 affine matrix of each
tetrahedron, not from the Jacobian route of ``oracle.geometry``):

* u = 0 (Stokes limit): only the pressure gradient term and the PSPG term
  remain, with the diffusive tau = (C_I nu^2 G:G)^{-1/2} constant per element;
* u constant, p linear: the SUPG term is (U . grad N_a) tau dp/dx_i with a
  constant tau = (U.G.U + C_I nu^2 G:G)^{-1/2}, the PSPG term grad N_a . grad p
  tau / rho;
* stabilisation switched off (C_I huge makes tau vanish): the Galerkin terms
  of eq. (NSt-weak) against the exact P1 mass matrix V(1 + delta_ab)/20
  (the convective integrand is linear per element), the textbook stiffness
  and the element divergence.

Flipping the sign or the weight of the SUPG or PSPG term in
``steady_residual`` fails the first two; a dropped or misweighted Galerkin
term fails the third.
"""
import numpy as np
import pytest

from oracle.steady import steady_residual
from workloads import cases, meshgen as mg


@pytest.fixture(scope="module")
def mesh():
    return mg.pipe(nc=2, nr=1, nz=3, seed=5)


def _affine_geometry(xyz, tets):
    """grad N_a [E,4,3], volume [E], metric G [E,3,3] from the inverse of
    [[1, x_a, y_a, z_a]]: column a of the inverse holds N_a's coefficients."""
    E = tets.shape[0]
    gradN = np.empty((E, 4, 3))
    vol = np.empty(E)
    for e in range(E):
        Mx = np.hstack([np.ones((4, 1)), xyz[tets[e]]])   # rows: vertices
        Minv = np.linalg.inv(Mx)                          # Minv[:, a] = (c0, cx, cy, cz) of N_a
        gradN[e] = Minv[1:, :].T
        vol[e] = abs(np.linalg.det(Mx)) / 6.0
    # G_ij = sum_k dxi_k/dx_i dxi_k/dx_j with xi_k = N_k (k = 1..3)
    G = np.einsum("eki,ekj->eij", gradN[:, 1:, :], gradN[:, 1:, :])
    return gradN, vol, G


def _mask(mesh):
    return cases.dirichlet_nodes(mesh, (mg.TAG_WALL, mg.TAG_INLET1))


def test_stokes_limit_pressure_and_pspg_terms(mesh):
    rng = np.random.default_rng(1)
    rho, mu, C_I = 1.7, 0.3, 3.0
    nu = mu / rho
    V = mesh.n_nodes
    dmask = _mask(mesh)
    p = rng.standard_normal(V)
    u = np.zeros((V, 3))
    Rm, Rc = steady_residual(mesh.xyz, mesh.tets, u, p, rho, mu, C_I, dmask)
    gradN, vol, G = _affine_geometry(mesh.xyz, mesh.tets)
    Em = np.zeros((V, 3))
    Ec = np.zeros(V)
    for e, t in enumerate(mesh.tets):
        gp = gradN[e].T @ p[t]
        tau = (C_I * nu * nu * np.sum(G[e] * G[e])) ** -0.5
        for a in range(4):
            Em[t[a]] += -vol[e] * gradN[e, a] * p[t].mean()
            Ec[t[a]] += vol[e] * tau / rho * (gradN[e, a] @ gp)
    Em[dmask] = 0.0
    np.testing.assert_allclose(Rm, Em, rtol=0, atol=1e-12 * np.abs(Em).max())
    np.testing.assert_allclose(Rc, Ec, rtol=0, atol=1e-12 * np.abs(Ec).max())
    assert np.abs(Ec).max() > 1e-3 * np.abs(Em).max()   # the PSPG term is not negligible here


def test_uniform_flow_linear_pressure_supg_pspg_closed_form(mesh):
    rho, mu, C_I = 1.3, 0.02, 3.0
    nu = mu / rho
    V = mesh.n_nodes
    dmask = _mask(mesh)
    U = np.array([0.4, -0.7, 1.1])
    gvec = np.array([0.3, 0.5, -0.9])
    u = np.tile(U, (V, 1))
    p = mesh.xyz @ gvec + 0.25
    Rm, Rc = steady_residual(mesh.xyz, mesh.tets, u, p, rho, mu, C_I, dmask)
    gradN, vol, G = _affine_geometry(mesh.xyz, mesh.tets)
    Em = np.zeros((V, 3))
    Ec = np.zeros(V)
    for e, t in enumerate(mesh.tets):
        tau = (U @ G[e] @ U + C_I * nu * nu * np.sum(G[e] * G[e])) ** -0.5
        pc = mesh.xyz[t].mean(axis=0) @ gvec + 0.25       # p at the centroid = mean of nodal p
        for a in range(4):
            Em[t[a]] += -vol[e] * gradN[e, a] * pc + vol[e] * (U @ gradN[e, a]) * tau * gvec
            Ec[t[a]] += vol[e] * tau / rho * (gradN[e, a] @ gvec)
    Em[dmask] = 0.0
    np.testing.assert_allclose(Rm, Em, rtol=0, atol=1e-12 * np.abs(Em).max())
    np.testing.assert_allclose(Rc, Ec, rtol=0, atol=1e-12 * np.abs(Ec).max())
    # the SUPG part carries a sizeable share of the momentum rows
    supg = np.zeros((V, 3))
    for e, t in enumerate(mesh.tets):
        tau = (U @ G[e] @ U + C_I * nu * nu * np.sum(G[e] * G[e])) ** -0.5
        for a in range(4):
            supg[t[a]] += vol[e] * (U @ gradN[e, a]) * tau * gvec
    supg[dmask] = 0.0
    assert np.abs(supg).max() > 1e-2 * np.abs(Em).max()


def test_galerkin_terms_with_stabilisation_switched_off(mesh):
    rng = np.random.default_rng(2)
    rho, mu = 0.9, 0.05
    V = mesh.n_nodes
    dmask = _mask(mesh)
    u = rng.standard_normal((V, 3))
    p = rng.standard_normal(V)
    # tau ~ 1e-20 of its usual size: SUPG and PSPG vanish below round-off
    Rm, Rc = steady_residual(mesh.xyz, mesh.tets, u, p, rho, mu, 1e40, dmask)
    gradN, vol, _ = _affine_geometry(mesh.xyz, mesh.tets)
    Em = np.zeros((V, 3))
    Ec = np.zeros(V)
    Mref = (np.ones((4, 4)) + np.eye(4)) / 20.0            # int N_a N_b / V
    for e, t in enumerate(mesh.tets):
        ue = u[t]                                           # [4, 3]
        gu = gradN[e].T @ ue                                # [j, i] = du_i/dx_j
        conv_nodes = ue @ gu                                # (u . grad) u at each vertex, [4, 3]
        for a in range(4):
            Em[t[a]] += rho * vol[e] * (Mref[a] @ conv_nodes)
            Em[t[a]] += -vol[e] * gradN[e, a] * p[t].mean()
            Em[t[a]] += mu * vol[e] * (gu.T @ gradN[e, a])
            Ec[t[a]] += 0.25 * vol[e] * np.trace(gu)
    Em[dmask] = 0.0
    np.testing.assert_allclose(Rm, Em, rtol=0, atol=1e-12 * np.abs(Em).max())
    np.testing.assert_allclose(Rc, Ec, rtol=0, atol=1e-12 * np.abs(Ec).max())
