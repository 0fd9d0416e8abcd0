"""Parity at the benchmark's full size, through the kernels the benchmark times.

Workload: the seeded Fontan-like cross junction (187,989 tets, 38,250 nodes),
N = 7, Re 500, Wo 10, resistance outlets, pseudo-time step 0.2: the FP64
residual (tau by the double-float refinement), the FP32 residual, and the
single-launch FP32 LIN_A tangent product after either residual.  The oracle
cannot evaluate the whole mesh in seconds, so each check compares the rows of
seeded sample nodes (interior, wall, inlet and outlet nodes); the oracle
computes those rows exactly from the elements that touch the sampled nodes,
and its outlet coupling uses the full state.  Bars as in test_gpu_parity:
relative L2 over the sampled rows <= 1e-12 (FP64) and <= 1e-5 (FP32).
"""
import math

import numpy as np
import pytest

from oracle import operator as op
from workloads import cases, meshgen as mg

from gpu_util import mass_coef, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

DT = 0.2


@pytest.fixture(scope="module")
def full():
    import torch
    import paper_2311_09465_gb300 as ts
    mesh = mg.junction(h=0.123, seed=1)
    case = cases.junction_case(N=7, Re=500.0, Wo=10.0, wave_seed=100, resistance=1.0, mesh=mesh, amp=0.05)
    y = case.y0 + 0.3 * cases.random_state(mesh, 7, seed=21)
    y[case.dirichlet_mask, 0:3] = case.y0[case.dirichlet_mask, 0:3]
    y[:, :, 0, 1] = 0.0
    v = cases.random_state(mesh, 7, seed=22, smooth=False)
    rng = np.random.default_rng(23)
    picks = [rng.choice(mesh.n_nodes, 16, replace=False)]
    for tag in (mg.TAG_WALL, mg.TAG_INLET1, mg.TAG_OUTLET1, mg.TAG_OUTLET2):
        pool = np.nonzero(cases.nodes_with_tag(mesh, tag))[0]
        picks.append(rng.choice(pool, 3, replace=False))
    nodes = np.unique(np.concatenate(picks))
    prob = op.problem_from_case(case)
    el = op.element_sample_for_nodes(prob, nodes)
    lin = op.linearize(prob, y, elems=el)
    r_ref = op.apply(prob, lin, y, "frozen")[nodes]
    hv_ref = op.apply(prob, lin, v, "lin_a", mask_dirichlet_input=True,
                      mass_coef=mass_coef(case, DT))[nodes]
    g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=DT)
    yield dict(torch=torch, case=case, y=y, v=v, nodes=nodes, r_ref=r_ref, hv_ref=hv_ref, g=g)
    g.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_fullsize_residual_rows(full, prec):
    torch = full["torch"]
    dty = torch.float64 if prec == 64 else torch.float32
    r = to_np(full["g"].residual(to_dev(full["y"], dty)))[full["nodes"]]
    err = rel_l2(r, full["r_ref"])
    print(f"full-size residual FP{prec}: rel L2 {err:.2e} over {len(full['nodes'])} nodes")
    assert err <= (1e-12 if prec == 64 else 1e-5), err


@pytest.mark.parametrize("state_prec", [64, 32])
def test_fullsize_fp32_tangent_rows(full, state_prec):
    # after an FP64 residual (the solver's path: state converted to FP32) or an FP32 one
    torch = full["torch"]
    g = full["g"]
    g.residual(to_dev(full["y"], torch.float64 if state_prec == 64 else torch.float32))
    hv = to_np(g.jvp(to_dev(full["v"], torch.float32)))[full["nodes"]]
    err = rel_l2(hv, full["hv_ref"])
    print(f"full-size FP32 LIN_A tangent after FP{state_prec} residual: rel L2 {err:.2e}")
    assert err <= 1e-5, err
    assert math.isfinite(float(np.abs(hv).max()))
