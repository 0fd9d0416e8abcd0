"""The exact tangent (TS_JVP_EXACT): the LIN_A product plus the derivative of
tau, d tau[v] L(u0), from the eigenpairs of M (Daleckii-Krein).

Pinned against the oracle without new oracle code: central differences of
the oracle's full residual (eq. Rmc, tau recomputed at every evaluation,
eq. 3D-tau), Richardson-extrapolated.  Bars: the FP32 product within 1e-5
relative L2 of the differences, and the tau-derivative term itself (exact
minus LIN_A) within 1e-2 of the differences' own tau part.
"""
import math

import numpy as np
import pytest

from oracle import operator as op
from workloads import cases, meshgen as mg

from gpu_util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _state(case, seed, scale=1.0):
    y = case.y0 + scale * cases.random_state(case.mesh, case.N, seed=seed)
    y[case.dirichlet_mask, 0:3] = case.y0[case.dirichlet_mask, 0:3]
    y[:, :, 0, 1] = 0.0
    return y


def _fd(prob, y, v):
    """Fourth-order central differences of the oracle residual along v."""
    eps = 1e-4 * np.linalg.norm(y) / np.linalg.norm(v)

    def d(h):
        return (op.residual(prob, y + h * v) - op.residual(prob, y - h * v)) / (2 * h)
    return (4.0 * d(eps / 2) - d(eps)) / 3.0


CASES = {
    "pipe_N3": lambda: cases.pipe_case(N=3, Re=150.0, Wo=5.0, mesh=mg.pipe(nc=2, nr=1, nz=3)),
    "junction_N4": lambda: cases.junction_case(N=4, Re=300.0, Wo=8.0, mesh=mg.junction(h=0.6, seed=3)),
    "pipe_N7": lambda: cases.pipe_case(N=7, Re=150.0, Wo=5.0, mesh=mg.pipe(nc=2, nr=2, nz=4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_exact_product_matches_central_differences_of_the_residual(name):
    import torch
    import paper_2311_09465_gb300 as ts
    case = CASES[name]()
    if name == "junction_N4":
        case.resistance = {mg.TAG_OUTLET1: 0.5}
    y = _state(case, seed=31, scale=0.8)
    v = cases.random_state(case.mesh, case.N, seed=32)
    v[case.dirichlet_mask, 0:3] = 0.0
    v[:, :, 0, 1] = 0.0
    prob = op.problem_from_case(case)
    fd = _fd(prob, y, v)
    lin_a = op.jvp(prob, op.linearize(prob, y), v, "lin_a")
    g = ts.GLSProblem(case, variant="exact", dt_pseudo=math.inf)
    g.residual(to_dev(y, torch.float64))
    got = to_np(g.jvp(to_dev(v, torch.float32)))
    assert rel_l2(got, fd) <= 1e-5, rel_l2(got, fd)
    # the tau derivative matters here, and the kernel's version of it is right
    dtau_fd = fd - lin_a
    assert np.linalg.norm(dtau_fd) > 1e-3 * np.linalg.norm(fd)
    assert np.linalg.norm((got - lin_a) - dtau_fd) <= 1e-2 * np.linalg.norm(dtau_fd)
    # the same product after an FP32 residual
    g.residual(to_dev(y, torch.float32))
    got32 = to_np(g.jvp(to_dev(v, torch.float32)))
    assert rel_l2(got32, fd) <= 1e-5, rel_l2(got32, fd)
    g.close()


def test_exact_tangent_needs_its_caches_and_fp32():
    import torch
    import paper_2311_09465_gb300 as ts
    case = CASES["pipe_N3"]()
    y = to_dev(_state(case, seed=33), torch.float64)
    g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=math.inf)
    g.residual(y)
    g.set(dt_pseudo=math.inf, variant="exact")
    with pytest.raises(ts.TsError) as ei:           # residual computed without the caches
        g.jvp(g.field(torch.float32))
    assert ei.value.code == ts.TS_ERR_ARG
    g.residual(y)
    with pytest.raises(ts.TsError) as ei:           # FP64 products are not provided
        g.jvp(g.field(torch.float64))
    assert ei.value.code == ts.TS_ERR_UNSUPPORTED
    g.close()


def test_exact_newton_converges_to_the_oracle_root():
    import torch
    import paper_2311_09465_gb300 as ts
    from oracle import solver as sv
    case = cases.pipe_case(N=3, Re=50.0, Wo=4.0, amps=(1.0, 0.5, 0.25), mesh=mg.pipe(nc=2, nr=1, nz=4))
    case.resistance = {mg.TAG_OUTLET1: 0.3}
    prob = op.problem_from_case(case)
    y_ref, rep_ref = sv.pseudo_time_solve(prob, case.y0, dt=math.inf, tol=1e-11, linear="gmres",
                                          eps_ls=0.05, variant="lin_a", max_steps=60)
    g = ts.GLSProblem(case, variant="exact", dt_pseudo=math.inf)
    y = to_dev(case.y0, torch.float64)
    rep = g.solve(y, precision=32, tol=1e-10, r_ref=rep_ref["r_ref"], max_steps=60, eps_ls=1e-4, precond=2)
    assert rep["r_final"] <= 1e-10
    assert rel_l2(to_np(y), y_ref) <= 1e-6
    # Newton with the exact derivative needs fewer steps than the tau-frozen one
    g2 = ts.GLSProblem(case, variant="lin_a", dt_pseudo=math.inf)
    y2 = to_dev(case.y0, torch.float64)
    rep2 = g2.solve(y2, precision=32, tol=1e-10, r_ref=rep_ref["r_ref"], max_steps=60, eps_ls=1e-4, precond=2)
    assert rep["steps"] <= rep2["steps"], (rep["steps"], rep2["steps"])
    g.close()
    g2.close()
