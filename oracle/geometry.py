"""Linear tetrahedron geometry: shape-function gradients, metric, quadrature.

Parent coordinates (a reading; the paper does not state them): the unit
reference tetrahedron, x = x_0 + sum_k xi_k (x_k - x_0), N_0 = 1 - xi_1 -
xi_2 - xi_3, N_k = xi_k.  Then d(xi)/dx = J^{-1} with J_{ik} = dx_i/dxi_k,
and the metric of eq. (metric) is G_ij = sum_k dxi_k/dx_i dxi_k/dx_j.

Quadrature (a reading of "each Gauss point", section 4): the symmetric
4-point rule of degree 2, weights V/4.

Pinned by: tests/test_oracle_geometry.py (gradients reproduce linear
functions exactly, partition of unity, volume of a known tetrahedron, the
rule integrates N_a N_b exactly).
"""
from __future__ import annotations

import numpy as np

_QA = 0.5854101966249685   # (5 + 3 sqrt 5) / 20
_QB = 0.1381966011250105   # (5 - sqrt 5) / 20
QP_BARY = np.array([
    [_QA, _QB, _QB, _QB],
    [_QB, _QA, _QB, _QB],
    [_QB, _QB, _QA, _QB],
    [_QB, _QB, _QB, _QA],
])                          # [q, a] = N_a at quadrature point q


def tet_geometry(xyz: np.ndarray, tets: np.ndarray):
    """Return dN [E,4,3] (dN_a/dx_i), vol [E], G [E,3,3]."""
    p = xyz[tets]                                  # [E,4,3]
    J = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)  # [E,i,k]
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                        # [E,k,i] = dxi_k/dx_i
    dN = np.empty((tets.shape[0], 4, 3))
    dN[:, 1:, :] = Jinv
    dN[:, 0, :] = -Jinv.sum(axis=1)
    G = np.einsum("eki,ekj->eij", Jinv, Jinv)
    vol = np.abs(detJ) / 6.0
    return dN, vol, G


def face_normals_areas(xyz: np.ndarray, faces: np.ndarray):
    """Unit outward normal [F,3] and area [F] of oriented boundary triangles."""
    a, b, c = xyz[faces[:, 0]], xyz[faces[:, 1]], xyz[faces[:, 2]]
    n = np.cross(b - a, c - a)
    area2 = np.linalg.norm(n, axis=1)
    return n / area2[:, None], 0.5 * area2
