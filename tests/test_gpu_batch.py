"""Batched lockstep solve (ts_batch_*): the fused multi-instance tangent
launch against each instance's own tangent product, and the lockstep
mixed-precision solve against the oracle and against one-by-one solves.

Bars: fused tangent within 2e-6 relative L2 of the single-instance FP32
kernel (both accumulate with atomics in different orders); converged fields
within 1e-6 of the one-by-one solves and of the FP64 oracle's solution.
"""
import math

import numpy as np
import pytest

from oracle import operator as op
from oracle import solver as sv
from workloads import cases, meshgen as mg

from gpu_util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _instances():
    """Uneven meshes and mode counts, each with its own waveform and Re."""
    out = []
    out.append(cases.pipe_case(N=3, Re=80.0, Wo=5.0, amps=(1.0, 0.4, 0.1), mesh=mg.pipe(nc=3, nr=2, nz=8)))
    c = cases.pipe_case(N=5, Re=120.0, Wo=4.0, amps=(1.0, 0.3j, 0.1, 0.05), mesh=mg.pipe(nc=2, nr=2, nz=10))
    c.resistance = {mg.TAG_OUTLET1: 0.5}
    out.append(c)
    out.append(cases.junction_case(N=4, Re=60.0, Wo=4.0, mesh=mg.junction(h=0.6, seed=3), amp=0.1))
    out.append(cases.pipe_case(N=7, Re=60.0, Wo=6.0, amps=(1.0, 0.2, 0.1, 0.05), mesh=mg.pipe(nc=2, nr=1, nz=6)))
    # small enough for the oracle's own solve
    c = cases.pipe_case(N=3, Re=50.0, Wo=4.0, amps=(1.0, 0.5, 0.25), mesh=mg.pipe(nc=2, nr=1, nz=4))
    c.resistance = {mg.TAG_OUTLET1: 0.3}
    out.append(c)
    return out


def test_fused_tangent_matches_single_instance(torch):
    import paper_2311_09465_gb300 as ts
    insts = _instances()
    gs = [ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.7) for c in insts]
    vs, ref = [], []
    for i, (c, g) in enumerate(zip(insts, gs)):
        y = c.y0 + 0.2 * cases.random_state(c.mesh, c.N, seed=20 + i)
        g.residual(to_dev(y, torch.float64))
        v = to_dev(cases.random_state(c.mesh, c.N, seed=40 + i), torch.float32)
        vs.append(v)
        ref.append(to_np(g.jvp(v)))
    b = ts.Batch(gs)
    out = b.jvp(vs)
    for o, r in zip(out, ref):
        assert rel_l2(to_np(o), r) <= 2e-6, rel_l2(to_np(o), r)
    b.close()
    for g in gs:
        g.close()


def test_batched_solve_matches_one_by_one_and_oracle(torch):
    import paper_2311_09465_gb300 as ts
    insts = _instances()
    opts = dict(tol=1e-9, max_steps=60, krylov=40, eps_ls=0.05, ser=1.0)
    single = []
    for c in insts:
        g = ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.5)
        y = to_dev(c.y0, torch.float64)
        rep = g.solve(y, precision=32, **opts)
        assert rep["status"] == 0
        single.append(to_np(y))
        g.close()
    gs = [ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.5) for c in insts]
    ys = [to_dev(c.y0, torch.float64) for c in insts]
    b = ts.Batch(gs)
    reps = b.solve(ys, **opts)
    shape = b.launch_shape()
    assert shape["tuned"] and shape["warps_per_block"] in (2, 4)
    for y, s, r in zip(ys, single, reps):
        assert r["r_final"] <= 1e-9
        assert rel_l2(to_np(y), s) <= 1e-6, rel_l2(to_np(y), s)
    # the smallest instance against the FP64 oracle's own solve
    c = insts[4]
    y_ref, rep = sv.pseudo_time_solve(op.problem_from_case(c), c.y0, dt=math.inf, tol=1e-11, linear="gmres",
                                      eps_ls=0.05, variant="lin_a", max_steps=60)
    assert rep["converged"]
    assert rel_l2(to_np(ys[4]), y_ref) <= 1e-6, rel_l2(to_np(ys[4]), y_ref)
    b.close()
    for g in gs:
        g.close()


def test_batch_rejects_unsupported_modes(torch):
    import paper_2311_09465_gb300 as ts
    c = cases.pipe_case(N=10, Re=50.0, Wo=4.0, mesh=mg.pipe(nc=2, nr=1, nz=4))
    g = ts.GLSProblem(c)
    with pytest.raises(ts.TsError) as e:
        ts.Batch([g])
    assert e.value.code == ts.TS_ERR_UNSUPPORTED
    g.close()
