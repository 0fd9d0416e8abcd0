"""Pin: the dense tangent of eq. (K_mat), built block by block, equals the
matrix-free products of oracle.operator on every column."""
import numpy as np
import pytest

from oracle import operator as op
from oracle.solver import dense_matrix
from workloads import cases, meshgen as mg


@pytest.mark.parametrize("variant", ["frozen", "paper"])
@pytest.mark.parametrize("N", [2, 3])
def test_dense_tangent_equals_products(variant, N):
    mesh = mg.pipe(nc=2, nr=1, nz=2, seed=1)
    dmask = cases.dirichlet_nodes(mesh, (mg.TAG_WALL, mg.TAG_INLET1))
    outlets = [(mesh.bfaces[mesh.btag == mg.TAG_OUTLET1], 0.8)]
    prob = op.make_problem(mesh.xyz, mesh.tets, N, 1.2, 0.03, 0.9, dmask, 3.0, outlets)
    y = cases.random_state(mesh, N, seed=2)
    lin = op.linearize(prob, y)
    mass = 2.5
    Hr = dense_matrix(prob, lin, variant, mass)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(y.shape)
        ref = op.jvp(prob, lin, v, variant, mass)
        got = (Hr @ v.ravel()).reshape(y.shape)
        np.testing.assert_allclose(got, ref, atol=1e-11 * np.abs(ref).max())
    # the products are linear: one column check with a unit vector
    free = op.free_mask(prob).ravel()
    k = np.nonzero(free)[0][17]
    e = np.zeros(free.size)
    e[k] = 1.0
    np.testing.assert_allclose(op.jvp(prob, lin, e.reshape(y.shape), variant, mass).ravel(),
                               Hr[:, k], atol=1e-12 * np.abs(Hr).max())
