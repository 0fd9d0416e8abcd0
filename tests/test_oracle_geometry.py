"""Pins for oracle.geometry (P1 gradients, metric, 4-point rule)."""
import numpy as np

from oracle.geometry import QP_BARY, tet_geometry
from workloads import meshgen as mg


def test_gradients_reproduce_linear_fields():
    m = mg.pipe(nc=2, nr=1, nz=3)
    dN, vol, G = tet_geometry(m.xyz, m.tets)
    x = m.xyz[m.tets]                       # [E,4,3]
    grad = np.einsum("eaj,eai->eij", dN, x)  # d x_i / d x_j
    np.testing.assert_allclose(grad, np.broadcast_to(np.eye(3), grad.shape), atol=1e-11)
    np.testing.assert_allclose(dN.sum(axis=1), 0, atol=1e-11)
    assert np.all(vol > 0)
    np.testing.assert_allclose(vol.sum(), np.sum(mg.signed_volumes(m.xyz, m.tets)), rtol=1e-12)


def test_reference_tet_metric_and_volume():
    s = 0.5
    xyz = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s]], float)
    dN, vol, G = tet_geometry(xyz, np.array([[0, 1, 2, 3]]))
    np.testing.assert_allclose(vol, [s ** 3 / 6])
    np.testing.assert_allclose(G[0], np.eye(3) / s ** 2)


def test_quadrature_exact_for_quadratics():
    # int N_a N_b = V (1 + delta_ab) / 20 on any tetrahedron
    M = np.einsum("qa,qb->ab", QP_BARY, QP_BARY) / 4.0
    np.testing.assert_allclose(M, (np.ones((4, 4)) + np.eye(4)) / 20.0, atol=1e-15)
    np.testing.assert_allclose(QP_BARY.sum(axis=1), 1.0)
