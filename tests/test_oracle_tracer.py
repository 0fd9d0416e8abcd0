"""Pins for oracle.tracer: the time-spectral GLS convection-diffusion residual
of eq. (3D-weak), section 2.2, checked against what the formulation and the
mathematics fix, not against itself."""
import numpy as np
import pytest

from oracle import tracer as tr
from workloads import cases, meshgen as mg

# the symmetric 4-point rule of degree 2 on a tetrahedron (barycentric)
QA, QB = (5 + 3 * 5 ** 0.5) / 20, (5 - 5 ** 0.5) / 20


@pytest.fixture(scope="module")
def mesh():
    return mg.pipe(nc=2, nr=1, nz=3, seed=7)


def _boundary_mask(mesh):
    m = np.zeros(mesh.n_nodes, dtype=bool)
    m[mesh.bfaces.ravel()] = True
    return m


def _random_modes(rng, shape, N, decay=1.0):
    """Random storage-layout modes [..., N, 2] of a real signal (Im of mode 0 zero)."""
    x = rng.standard_normal(shape + (N, 2))
    x *= (1.0 / (1.0 + decay * np.arange(N)) ** 2)[:, None]
    x[..., 0, 1] = 0.0
    return x


def _tet_grads(p):
    """dN_a/dx (4 x 3) and volume of one tetrahedron, from its edge matrix."""
    J = np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]], axis=1)
    Jinv = np.linalg.inv(J)
    dN = np.vstack([-Jinv.sum(axis=0), Jinv])
    return dN, abs(np.linalg.det(J)) / 6.0


def test_one_mode_equals_steady_supg_gls_residual(mesh):
    # N = 1: A_i = a_i (scalar), Omega = 0, tau = (a.G.a + C_I kappa^2 G:G)^(-1/2): the
    # classical steady residual sum_q w [N_A a.grad phi + kappa grad N_A.grad phi
    # + tau (a.grad N_A)(a.grad phi)], written out element by element and point by point
    rng = np.random.default_rng(1)
    kappa, C_I = 0.07, 3.0
    dmask = _boundary_mask(mesh)
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, 1, kappa, 0.9, dmask, C_I)
    a = _random_modes(rng, (mesh.n_nodes, 3), 1)
    phi = _random_modes(rng, (mesh.n_nodes,), 1)
    got = tr.tracer_residual(tp, a, phi)[:, 0, 0]
    ref = np.zeros(mesh.n_nodes)
    for tet in mesh.tets:
        p = mesh.xyz[tet]
        dN, vol = _tet_grads(p)
        Jinv = dN[1:]                      # [k, i] = dxi_k/dx_i, unit reference tetrahedron
        G = Jinv.T @ Jinv                  # G_ij = sum_k dxi_k/dx_i dxi_k/dx_j (eq. metric)
        gphi = dN.T @ phi[tet, 0, 0]
        for q in range(4):
            lam = np.full(4, QB)
            lam[q] = QA
            av = lam @ a[tet, :, 0, 0]
            tau = (av @ G @ av + C_I * kappa ** 2 * np.sum(G * G)) ** -0.5
            adv = av @ gphi
            for A in range(4):
                ref[tet[A]] += vol / 4 * (lam[A] * adv + kappa * dN[A] @ gphi
                                          + tau * (av @ dN[A]) * adv)
    ref[dmask] = 0.0
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


def test_no_velocity_one_mode_is_kappa_times_stiffness(mesh):
    # a = 0, N = 1: res(phi) = 0 on P1 elements, only kappa (grad N_A, grad N_B) phi_B remains
    rng = np.random.default_rng(2)
    kappa = 0.3
    dmask = _boundary_mask(mesh)
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, 1, kappa, 1.0, dmask)
    phi = _random_modes(rng, (mesh.n_nodes,), 1)
    got = tr.tracer_residual(tp, np.zeros((mesh.n_nodes, 3, 1, 2)), phi)[:, 0, 0]
    K = np.zeros((mesh.n_nodes, mesh.n_nodes))
    for tet in mesh.tets:
        dN, vol = _tet_grads(mesh.xyz[tet])
        K[np.ix_(tet, tet)] += vol * dN @ dN.T
    ref = kappa * K @ phi[:, 0, 0]
    ref[dmask] = 0.0
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


def test_conjugate_symmetry_and_real_mode0(mesh):
    # real velocity and tracer signals give r_{-m} = conj(r_m) and Im r_0 = 0
    rng = np.random.default_rng(3)
    N = 4
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, N, 0.05, 0.8, _boundary_mask(mesh))
    a = _random_modes(rng, (mesh.n_nodes, 3), N)
    a[:, :, 0, 0] += 1.5
    phi = _random_modes(rng, (mesh.n_nodes,), N)
    rc = tr.tracer_residual(tp, a, phi, return_complex=True)
    s = np.abs(rc).max()
    np.testing.assert_allclose(rc[:, : N - 1], np.conj(rc[:, N:][:, ::-1]), atol=1e-12 * s)
    assert np.abs(rc[:, N - 1].imag).max() < 1e-12 * s


def test_linear_field_across_uniform_flow_is_an_exact_solution(mesh):
    # a(t) uniform in space along x (three modes), phi = y + 2 z steady: a.grad phi = 0,
    # Omega phi = 0 and the P1 Laplacian of a linear field vanishes row by row, so
    # every equation (interior row) is satisfied exactly
    N = 3
    interior = ~_boundary_mask(mesh)
    assert interior.sum() > 0
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, N, 0.04, 1.3, ~interior)
    a = np.zeros((mesh.n_nodes, 3, N, 2))
    a[:, 0, 0, 0], a[:, 0, 1, 0], a[:, 0, 1, 1], a[:, 0, 2, 0] = 1.0, 0.4, -0.2, 0.1
    phi = np.zeros((mesh.n_nodes, N, 2))
    phi[:, 0, 0] = mesh.xyz[:, 1] + 2.0 * mesh.xyz[:, 2]
    r = tr.tracer_residual(tp, a, phi)
    assert np.abs(r[interior]).max() < 1e-12 * np.abs(phi).max()
    # a field along the flow is not a solution (the check has teeth)
    phi[:, 0, 0] = mesh.xyz[:, 0]
    assert np.abs(tr.tracer_residual(tp, a, phi)[interior]).max() > 1e-3


def test_energy_identity_for_uniform_flow(mesh):
    # Lemma-1-type identity: a uniform in space (time-periodic) and phi = 0 on the boundary
    # give Re(phi^H r(phi)) = kappa |grad phi|^2 + sum_q w res^H tau res: the Galerkin
    # convective term sum_i (phi, A_i dphi/dx_i) and (phi, Omega phi) are purely imaginary
    from oracle.spectral import conv_matrix, omega_diag, to_complex
    from oracle.tau import tau_matrix
    rng = np.random.default_rng(4)
    N, kappa, omega, C_I = 3, 0.06, 0.9, 3.0
    bmask = _boundary_mask(mesh)
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, N, kappa, omega, bmask, C_I)
    a1 = _random_modes(rng, (3,), N)
    a1[:, 0, 0] += np.array([1.0, -0.5, 0.3])
    a = np.broadcast_to(a1, (mesh.n_nodes, 3, N, 2)).copy()
    phi = _random_modes(rng, (mesh.n_nodes,), N)
    phi[bmask] = 0.0
    r = tr.tracer_residual(tp, a, phi, return_complex=True)
    Phi = to_complex(phi, N)
    lhs = np.real(np.sum(np.conj(Phi) * r))
    # right side from the pieces, element by element
    A = conv_matrix(to_complex(a1, N))                # [3, nm, nm], the same at every point
    om = omega_diag(N, omega)
    rhs = 0.0
    for tet in mesh.tets:
        dN, vol = _tet_grads(mesh.xyz[tet])
        Jinv = dN[1:]
        G = Jinv.T @ Jinv
        tau = tau_matrix(A, G, kappa, C_I)
        g = dN.T @ Phi[tet]                            # [3, nm]
        rhs += kappa * vol * np.sum(np.abs(g) ** 2)
        for q in range(4):
            lam = np.full(4, QB)
            lam[q] = QA
            res = om * (lam @ Phi[tet]) + np.einsum("jmn,jn->m", A, g)
            rhs += vol / 4 * np.real(np.conj(res) @ tau @ res)
    assert rhs > 0
    assert abs(lhs - rhs) <= 1e-11 * rhs
