"""Block preconditioners vs the oracle (ts_block_diagonal; ts_solve precond = 2 and 3).

* Blocks: the oracle's dense tangent (eq. K_mat, assembled block by block,
  ``oracle.assemble``) restricted to each node's own unknowns equals the
  library's H_AA for every node, FROZEN and PAPER variants, with and without
  the pseudo-time mass, with a resistance outlet; FP32 bar 1e-5 relative L2.
* Inverse: the stored inverse times H_AA (fixed rows and columns set to the
  identity) is the identity.
* Applications (ts_precond_apply): block Jacobi and the forward-backward
  block Gauss-Seidel sweeps equal the same block operations done in FP64 on
  the oracle's dense tangent in the library's node-colour order; FP32 bar
  1e-4 relative L2.
* Solve: with the nodal block-Jacobi (precond 2) or the symmetric block
  Gauss-Seidel (precond 3) preconditioner the solve reaches the oracle's root
  within the converged-field bar 1e-6 (pipe: the oracle's own solve; small
  Re-300 junction: the oracle field written by tests/golden/make_junction_re300.py).
"""
import math
import os
import sys

import numpy as np
import pytest

from oracle import operator as op
from oracle import precond as pc
from oracle import solver as sv
from workloads import cases, meshgen as mg

from gpu_util import mass_coef, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _state(case, seed, scale=1.0):
    y = case.y0 + scale * cases.random_state(case.mesh, case.N, seed=seed)
    y[case.dirichlet_mask, 0:3] = case.y0[case.dirichlet_mask, 0:3]
    y[:, :, 0, 1] = 0.0
    return y


def _pipe(N, **kw):
    c = cases.pipe_case(N=N, Re=120.0, Wo=5.0, mesh=mg.pipe(**kw))
    c.resistance = {mg.TAG_OUTLET1: 0.6}
    return c


BLOCK_CASES = [
    ("pipe_N1", lambda: _pipe(1, nc=2, nr=1, nz=3), "frozen", math.inf, 64),
    ("pipe_N3", lambda: _pipe(3, nc=2, nr=1, nz=3), "frozen", 0.7, 64),
    ("pipe_N3_paper", lambda: _pipe(3, nc=2, nr=1, nz=3), "paper", math.inf, 64),
    ("pipe_N4_fp32", lambda: _pipe(4, nc=2, nr=1, nz=2), "frozen", 0.7, 32),
    ("pipe_N7", lambda: _pipe(7, nc=2, nr=1, nz=2), "lin_a", 1.3, 64),
]


@pytest.mark.parametrize("name,make,variant,dt,prec", BLOCK_CASES, ids=[c[0] for c in BLOCK_CASES])
def test_block_diagonal_matches_dense_tangent(name, make, variant, dt, prec):
    import torch
    import paper_2311_09465_gb300 as ts
    case = make()
    y = _state(case, seed=5, scale=0.8)
    N, V = case.N, case.mesh.n_nodes
    nb = 8 * N
    prob = op.problem_from_case(case)
    lin = op.linearize(prob, y)
    # a LIN_A problem's blocks are those of the frozen tangent
    Hr = sv.dense_matrix(prob, lin, "paper" if variant == "paper" else "frozen", mass_coef(case, dt))
    Hr = Hr.reshape(V, nb, V, nb)
    ref = np.stack([Hr[A, :, A, :] for A in range(V)])
    g = ts.GLSProblem(case, variant=variant, dt_pseudo=dt)
    g.residual(to_dev(y, torch.float64 if prec == 64 else torch.float32))
    got = to_np(g.block_diagonal(invert=False))
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)
    # the inverse (column-major) undoes the block with fixed unknowns set to the identity
    inv = to_np(g.block_diagonal(invert=True)).transpose(0, 2, 1)
    fixed = np.zeros((V, 4, N, 2), dtype=bool)
    fixed[:, :, 0, 1] = True
    fixed[case.dirichlet_mask, 0:3] = True
    fixed = fixed.reshape(V, nb)
    B = got.copy()
    for A in range(V):
        B[A][fixed[A], :] = 0.0
        B[A][:, fixed[A]] = 0.0
        B[A][fixed[A], fixed[A]] = 1.0
    eye = np.eye(nb)
    worst = max(np.linalg.norm(inv[A] @ B[A] - eye) / math.sqrt(nb) for A in range(V))
    assert worst <= 1e-4, worst
    g.close()


def _fixed_mask(case):
    V, N = case.mesh.n_nodes, case.N
    fixed = np.zeros((V, 4, N, 2), dtype=bool)
    fixed[:, :, 0, 1] = True
    fixed[case.dirichlet_mask, 0:3] = True
    return fixed.reshape(V, 8 * N)


SWEEP_CASES = [
    ("pipe_N3_paper", lambda: _pipe(3, nc=2, nr=2, nz=4), "paper", 0.8),
    ("pipe_N3_lin_a", lambda: _pipe(3, nc=2, nr=1, nz=5), "lin_a", 0.4),
    ("pipe_N7_lin_a", lambda: _pipe(7, nc=2, nr=1, nz=3), "lin_a", 1.3),
]


@pytest.mark.parametrize("name,make,variant,dt", SWEEP_CASES, ids=[c[0] for c in SWEEP_CASES])
def test_preconditioner_applications_match_dense_block_sweeps(name, make, variant, dt):
    """ts_precond_apply kind 2 and 3 against the same block operations on the
    oracle's dense tangent (eq. K_mat): on the diagonal the blocks of the
    problem's variant (FROZEN for LIN_A), off it the paper variant's
    (section 2.5.2), the sweeps in the library's node-colour order.  No
    resistance outlet: its coupling between different nodes is left out of
    the Gauss-Seidel blocks by design.  FP32 bar 1e-4 relative L2."""
    import torch
    import paper_2311_09465_gb300 as ts
    case = make()
    case.resistance = {}
    y = _state(case, seed=7, scale=0.8)
    N, V = case.N, case.mesh.n_nodes
    nb = 8 * N
    prob = op.problem_from_case(case)
    lin = op.linearize(prob, y)
    mc = mass_coef(case, dt)
    Hd = sv.dense_matrix(prob, lin, "paper" if variant == "paper" else "frozen", mc).reshape(V, nb, V, nb)
    Hp = sv.dense_matrix(prob, lin, "paper", mc).reshape(V, nb, V, nb)
    fixed = _fixed_mask(case)
    Dinv, _ = pc.masked_blocks(Hd, fixed)
    _, off = pc.masked_blocks(Hp, fixed)
    x = cases.random_state(case.mesh, N, seed=8).reshape(V, nb)
    x[fixed] = 0.0

    g = ts.GLSProblem(case, variant=variant, dt_pseudo=dt)
    g.residual(to_dev(y, torch.float64))
    xd = to_dev(x.reshape(V, 4, N, 2), torch.float64)
    with pytest.raises(ts.TsError):
        g.precond_apply(3, xd)
    # block Jacobi
    g.precond_setup(2)
    zj = to_np(g.precond_apply(2, xd)).reshape(V, nb)
    ref_j = pc.block_jacobi(Dinv, x)
    assert rel_l2(zj, ref_j) <= 1e-4, rel_l2(zj, ref_j)
    # symmetric block Gauss-Seidel over the node colours
    g.precond_setup(3)
    zs = to_np(g.precond_apply(3, xd)).reshape(V, nb)
    n_col, colour = g.node_colours()
    assert colour.shape == (V,) and colour.min() == 0 and colour.max() == n_col - 1
    assert pc.check_colouring(Hp, colour)   # a colour holds no two nodes of one element
    z = pc.symmetric_block_gauss_seidel(Dinv, off, colour, x)
    assert rel_l2(zs, z) <= 1e-4, rel_l2(zs, z)
    assert np.all(zs[fixed] == 0.0)
    # a new residual invalidates both
    g.residual(to_dev(y, torch.float64))
    with pytest.raises(ts.TsError):
        g.precond_apply(2, xd)
    g.close()


@pytest.fixture(scope="module")
def pipe_case():
    case = cases.pipe_case(N=3, Re=50.0, Wo=4.0, amps=(1.0, 0.5, 0.25), mesh=mg.pipe(nc=2, nr=1, nz=4))
    case.resistance = {mg.TAG_OUTLET1: 0.3}
    return case


@pytest.fixture(scope="module")
def pipe_solution(pipe_case):
    prob = op.problem_from_case(pipe_case)
    y, rep = sv.pseudo_time_solve(prob, pipe_case.y0, dt=math.inf, tol=1e-11, linear="gmres",
                                  eps_ls=0.05, variant="lin_a", max_steps=60)
    assert rep["converged"]
    return y, rep


@pytest.mark.parametrize("precision,precond", [(64, 2), (32, 2), (32, 3)])
def test_block_preconditioned_solve_matches_oracle_pipe(pipe_case, pipe_solution, precision, precond):
    import torch
    import paper_2311_09465_gb300 as ts
    y_ref, rep_ref = pipe_solution
    g = ts.GLSProblem(pipe_case, variant="lin_a", dt_pseudo=math.inf)
    y = to_dev(pipe_case.y0, torch.float64)
    rep = g.solve(y, precision=precision, tol=1e-10, r_ref=rep_ref["r_ref"], max_steps=100, precond=precond)
    got = to_np(y)
    assert rep["r_final"] <= 1e-10
    assert rel_l2(got, y_ref) <= 1e-6, rel_l2(got, y_ref)
    np.testing.assert_array_equal(got[pipe_case.dirichlet_mask, 0:3],
                                  pipe_case.y0[pipe_case.dirichlet_mask, 0:3])
    assert np.all(got[:, :, 0, 1] == 0)
    g.close()


def _golden_junction():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    try:
        import make_junction_re300 as mk
    finally:
        sys.path.pop(0)
    data = np.load(os.path.join(HERE, "golden", "junction_re300_N3.npz"))
    return mk.case(), data


@pytest.mark.parametrize("precision,precond", [(32, 2), (64, 2), (32, 3)])
def test_block_preconditioned_solve_matches_oracle_junction_re300(precision, precond):
    import torch
    import paper_2311_09465_gb300 as ts
    case, data = _golden_junction()
    assert int(data["n_tets"]) == case.mesh.n_tets
    g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=0.5)
    y = to_dev(case.y0, torch.float64)
    r_ref = float(data["r_ref"])
    rep = g.solve(y, precision=precision, tol=1e-10, r_ref=r_ref, max_steps=120, precond=precond, ser=1.0,
                  dt_max=1e6)
    assert rep["r_final"] <= 1e-10, rep["hist"][-5:]
    got = to_np(y)
    assert rel_l2(got, data["y"]) <= 1e-6, rel_l2(got, data["y"])
    # the oracle agrees that the GPU field is a root
    prob = op.problem_from_case(case)
    assert np.linalg.norm(op.residual(prob, got)) <= 1e-9 * r_ref
    g.close()
