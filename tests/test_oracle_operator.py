"""Pins for oracle.operator: eq. (Rmc) residual and eq. (K_mat) products."""
import numpy as np
import pytest

from oracle import operator as op
from oracle.steady import steady_residual
from workloads import cases, meshgen as mg


@pytest.fixture(scope="module")
def small():
    mesh = mg.pipe(nc=2, nr=1, nz=3, seed=5)
    return mesh


def _prob(mesh, N, omega=0.6, rho=1.1, mu=0.05, resistance=None):
    dmask = cases.dirichlet_nodes(mesh, (mg.TAG_WALL, mg.TAG_INLET1))
    outlets = [(mesh.bfaces[mesh.btag == mg.TAG_OUTLET1], resistance)] if resistance else []
    return op.make_problem(mesh.xyz, mesh.tets, N, rho, mu, omega, dmask, 3.0, outlets)


def test_steady_limit_equals_time_formulation_supg_pspg(small):
    # omega = 0, only mode 0 nonzero: eq. (NS-weak) reduces to eq. (NSt-weak) (App. B)
    rng = np.random.default_rng(0)
    for N in (1, 3):
        prob = _prob(small, N, omega=0.0)
        y = np.zeros((small.n_nodes, 4, N, 2))
        y[:, :, 0, 0] = cases.random_state(small, 1, seed=11)[:, :, 0, 0]
        r = op.residual(prob, y)
        Rm, Rc = steady_residual(small.xyz, small.tets, y[:, 0:3, 0, 0], y[:, 3, 0, 0],
                                 prob.rho, prob.mu, prob.C_I, prob.dmask)
        np.testing.assert_allclose(r[:, 0:3, 0, 0], Rm, atol=1e-12 * np.abs(Rm).max())
        np.testing.assert_allclose(r[:, 3, 0, 0], Rc, atol=1e-12 * np.abs(Rc).max())
        if N > 1:
            assert np.abs(r[:, :, 1:]).max() == 0.0
        assert np.abs(r[:, :, 0, 1]).max() == 0.0


def test_residual_conjugate_symmetry_and_real_mode0(small):
    # real data: r_{-m} = conj(r_m) and Im r_0 = 0 (section 3.3)
    N = 4
    prob = _prob(small, N, resistance=0.7)
    y = cases.random_state(small, N, seed=3)
    rc = op.residual(prob, y, return_complex=True)
    scale = np.abs(rc).max()
    np.testing.assert_allclose(rc[..., : N - 1], np.conj(rc[..., N:][..., ::-1]), atol=1e-12 * scale)
    assert np.abs(rc[..., N - 1].imag).max() < 1e-12 * scale


def test_frozen_product_equals_central_difference_at_rest(small):
    # at u = 0, A = 0 and tau is constant to O(eps^2): r(eps v) - r(-eps v) = 2 eps H v + O(eps^3)
    N = 3
    prob = _prob(small, N, resistance=0.5)
    y0 = np.zeros((small.n_nodes, 4, N, 2))
    v = cases.random_state(small, N, seed=4)
    v[prob.dmask, 0:3] = 0.0
    lin = op.linearize(prob, y0)
    Hv = op.jvp(prob, lin, v, "frozen")
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        fd = (op.residual(prob, eps * v) - op.residual(prob, -eps * v)) / (2 * eps)
        errs.append(np.abs(fd - Hv).max() / np.abs(Hv).max())
    # second-order agreement: the remainder comes from d2 tau / du2 only
    assert errs[2] < 1e-6
    assert 50 < errs[0] / errs[1] < 200


def test_pressure_columns_are_exact_derivative_at_any_state(small):
    # A and tau do not depend on p, so r is affine in p at fixed u
    N = 3
    prob = _prob(small, N, resistance=0.5)
    y = cases.random_state(small, N, seed=5)
    vp = np.zeros_like(y)
    vp[:, 3] = cases.random_state(small, N, seed=6)[:, 3]
    lin = op.linearize(prob, y)
    Hv = op.jvp(prob, lin, vp, "frozen")
    for eps in (1e-3, 1.0):
        fd = (op.residual(prob, y + eps * vp) - op.residual(prob, y)) / eps
        np.testing.assert_allclose(fd, Hv, atol=1e-9 * np.abs(Hv).max())


def test_paper_variant_differs_from_frozen_only_in_G_and_D(small):
    N = 3
    prob = _prob(small, N)
    y = cases.random_state(small, N, seed=7)
    lin = op.linearize(prob, y)
    vu = cases.random_state(small, N, seed=8)
    vu[:, 3] = 0.0
    vp = np.zeros_like(vu)
    vp[:, 3] = cases.random_state(small, N, seed=9)[:, 3]
    a = op.jvp(prob, lin, vu, "paper")
    b = op.jvp(prob, lin, vu, "frozen")
    # velocity input: momentum rows identical (K), continuity rows differ (D's LS part)
    np.testing.assert_allclose(a[:, 0:3], b[:, 0:3], atol=1e-12 * np.abs(b).max())
    assert np.abs(a[:, 3] - b[:, 3]).max() > 1e-6 * np.abs(b).max()
    a = op.jvp(prob, lin, vp, "paper")
    b = op.jvp(prob, lin, vp, "frozen")
    # pressure input: continuity rows identical (L), momentum rows differ (G's LS part)
    np.testing.assert_allclose(a[:, 3], b[:, 3], atol=1e-12 * np.abs(b).max())
    assert np.abs(a[:, 0:3] - b[:, 0:3]).max() > 1e-6 * np.abs(b).max()


def test_sampled_elements_reproduce_full_operator_at_sample_nodes(small):
    N = 2
    prob = _prob(small, N, resistance=0.3)
    y = cases.random_state(small, N, seed=10)
    full = op.residual(prob, y)
    nodes = np.array([0, 7, 19, small.n_nodes - 1])
    el = op.element_sample_for_nodes(prob, nodes)
    part = op.residual(prob, y, elems=el)
    np.testing.assert_allclose(part[nodes], full[nodes], atol=1e-13 * np.abs(full).max())


def test_lin_a_product_is_exact_derivative_with_tau_held(small):
    # with tau fixed the residual is a cubic polynomial in y (the least-squares
    # test function A_j(y) multiplies tau L(y)), so central differences converge
    # at second order with no other remainder
    N = 3
    prob = _prob(small, N, resistance=0.4)
    y = cases.random_state(small, N, seed=12)
    v = cases.random_state(small, N, seed=13)
    v[prob.dmask, 0:3] = 0.0
    lin = op.linearize(prob, y)
    Jv = op.jvp(prob, lin, v, "lin_a")

    def r_tau_held(z):
        return op.apply(prob, op.linearize(prob, z, tau_state=y), z, "frozen")

    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        fd = (r_tau_held(y + eps * v) - r_tau_held(y - eps * v)) / (2 * eps)
        errs.append(np.abs(fd - Jv).max() / np.abs(Jv).max())
    assert errs[2] < 1e-8
    assert 80 < errs[0] / errs[1] < 120 and 80 < errs[1] / errs[2] < 120
    # the 'frozen' product misses the dA/du terms by far more than that
    Jf = op.jvp(prob, lin, v, "frozen")
    assert np.abs(Jf - Jv).max() > 1e-3 * np.abs(Jv).max()
