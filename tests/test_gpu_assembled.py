"""Assembled block-structured tangent (ts_assemble, ts_spmv) vs the oracle.

Section 2.5.2 stores the tangent of eq. (K_mat) block by block with the
least-squares parts of G_i and D_j dropped; its product must equal the
paper-variant tangent product.  Bar: FP32 relative L2 1e-5 against the FP64
oracle's product on the same seeded state and input (with the pseudo-time
mass and a resistance outlet), and agreement with the library's own
matrix-free FP32 product of the same variant.
"""
import math

import numpy as np
import pytest

from oracle import operator as op
from workloads import cases, meshgen as mg

from gpu_util import mass_coef, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _state(case, seed, scale=1.0):
    y = case.y0 + scale * cases.random_state(case.mesh, case.N, seed=seed)
    y[case.dirichlet_mask, 0:3] = case.y0[case.dirichlet_mask, 0:3]
    y[:, :, 0, 1] = 0.0
    return y


def _pipe(N, **kw):
    c = cases.pipe_case(N=N, Re=100.0, Wo=5.0, mesh=mg.pipe(**kw))
    c.resistance = {mg.TAG_OUTLET1: 0.4}
    return c


CASES = [
    ("pipe_N1", lambda: _pipe(1, nc=2, nr=1, nz=3), math.inf),
    ("pipe_N3", lambda: _pipe(3, nc=2, nr=2, nz=4), 0.8),
    ("junction_N4", lambda: cases.junction_case(N=4, Re=300.0, Wo=8.0, mesh=mg.junction(h=0.6, seed=3)), 0.5),
    ("pipe_N7", lambda: _pipe(7, nc=2, nr=2, nz=4), 2.0),
    ("pipe_N15", lambda: _pipe(15, nc=2, nr=1, nz=2), 1.0),
]


@pytest.mark.parametrize("name,make,dt", CASES, ids=[c[0] for c in CASES])
def test_assembled_product_matches_oracle_paper_tangent(name, make, dt):
    import torch
    import paper_2311_09465_gb300 as ts
    case = make()
    y = _state(case, seed=11, scale=0.7)
    v = cases.random_state(case.mesh, case.N, seed=12)
    prob = op.problem_from_case(case)
    lin = op.linearize(prob, y)
    ref = op.jvp(prob, lin, v, "paper", mass_coef(case, dt))
    g = ts.GLSProblem(case, variant="paper", dt_pseudo=dt)
    g.residual(to_dev(y, torch.float64))
    g.assemble()
    v32 = to_dev(v, torch.float32)
    got = to_np(g.spmv(v32))
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    # the matrix-free product of the same variant
    mf = to_np(g.jvp(v32))
    assert rel_l2(got, mf) <= 1e-5, rel_l2(got, mf)
    # storage: K and L per connection plus six scalars
    C = 2 * case.N
    nnz = ts.ts_mesh_connections(g.mesh)
    assert g.assembled_bytes() == nnz * (2 * C * C + 8) * 4
    g.close()


def test_assembled_product_is_invalidated_by_a_new_residual():
    import torch
    import paper_2311_09465_gb300 as ts
    case = _pipe(3, nc=2, nr=1, nz=3)
    g = ts.GLSProblem(case, variant="paper", dt_pseudo=1.0)
    y = to_dev(_state(case, seed=1), torch.float64)
    g.residual(y)
    g.assemble()
    g.residual(y)
    with pytest.raises(ts.TsError) as ei:
        g.spmv(g.field(torch.float32))
    assert ei.value.code == ts.TS_ERR_ARG
    g.close()
