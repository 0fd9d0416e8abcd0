"""Converged fields of the GPU pseudo-time Newton-GMRES solve vs the oracle.

Bar: converged modal fields within relative L2 1e-6 of the FP64 oracle's
converged field on the same seeded case; the oracle's own residual of the
GPU field is at the solve tolerance.
"""
import math

import numpy as np
import pytest

from oracle import operator as op
from oracle import solver as sv
from oracle import womersley as wo
from workloads import cases, meshgen as mg

from gpu_util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipe_case():
    case = cases.pipe_case(N=3, Re=50.0, Wo=4.0, amps=(1.0, 0.5, 0.25), mesh=mg.pipe(nc=2, nr=1, nz=4))
    case.resistance = {mg.TAG_OUTLET1: 0.3}
    return case


@pytest.fixture(scope="module")
def oracle_solution(pipe_case):
    prob = op.problem_from_case(pipe_case)
    y, rep = sv.pseudo_time_solve(prob, pipe_case.y0, dt=math.inf, tol=1e-11, linear="gmres",
                                  eps_ls=0.05, variant="lin_a", max_steps=60)
    assert rep["converged"]
    return y, rep


@pytest.mark.parametrize("precision,variant,dt,precond", [(64, "lin_a", math.inf, 1),
                                                          (32, "lin_a", math.inf, 1),
                                                          (64, "paper", 2.0, 1),
                                                          (32, "frozen", math.inf, 0)])
def test_solve_matches_oracle(pipe_case, oracle_solution, precision, variant, dt, precond):
    import torch
    import paper_2311_09465_gb300 as ts
    y_ref, rep_ref = oracle_solution
    g = ts.GLSProblem(pipe_case, variant=variant, dt_pseudo=dt)
    y = to_dev(pipe_case.y0, torch.float64)
    rep = g.solve(y, precision=precision, tol=1e-10, r_ref=rep_ref["r_ref"], max_steps=300,
                  precond=precond)
    got = to_np(y)
    assert rep["r_final"] <= 1e-10
    assert rel_l2(got, y_ref) <= 1e-6, rel_l2(got, y_ref)
    # the oracle agrees that the GPU field is a root
    prob = op.problem_from_case(pipe_case)
    assert np.linalg.norm(op.residual(prob, got)) <= 1e-9 * rep_ref["r_ref"]
    # Dirichlet values untouched, Im(mode 0) zero
    np.testing.assert_array_equal(got[pipe_case.dirichlet_mask, 0:3],
                                  pipe_case.y0[pipe_case.dirichlet_mask, 0:3])
    assert np.all(got[:, :, 0, 1] == 0)


def test_womersley_pipe_config_closed_form():
    """Pipe of radius 1, length 5, N = 3, Re 100, Wo 5 (the plain-method FP64 case)."""
    import torch
    import paper_2311_09465_gb300 as ts
    case = cases.pipe_case(N=3, Re=100.0, Wo=5.0, amps=(1.0, 0.5, 0.25), mesh=mg.pipe(nc=4, nr=4, nz=20))
    # plain Newton diverges from the cold start at Re 100; pseudo-time with a
    # step that grows as the residual falls converges in about 13 steps
    g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=0.5)
    y = to_dev(case.y0, torch.float64)
    rep = g.solve(y, precision=64, tol=1e-8, max_steps=40, ser=1.0)
    assert rep["r_final"] <= 1e-8
    got = to_np(y)
    ex = wo.pipe_solution(case.mesh.xyz, case.info["R"], case.info["L"], case.info["U"],
                          case.rho, case.mu, case.omega)
    z = case.mesh.xyz[:, 2]
    sel = (z > 1.0) & (z < 4.0)
    err = rel_l2(got[sel, 0:3], ex[sel, 0:3])
    assert err < 0.08, err
    # the oracle's residual of the GPU field (full mesh, N = 3)
    prob = op.problem_from_case(case)
    assert np.linalg.norm(op.residual(prob, got)) <= 2e-8 * rep["r_ref"]
