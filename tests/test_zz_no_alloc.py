"""The allocation-free residual entry point (ts_residual_noalloc).

It serves callers that cannot allocate device memory at call time; it must
give the same residual as ts_residual in FP32, on repeated calls that reuse
its fixed scratch array, and refuse meshes too large for that array.  This
file is collected last so that a failure here stops a -x run only after all
other tests have run.
"""
import numpy as np
import pytest

from workloads import cases, meshgen as mg

from gpu_util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _state(case, seed):
    y = case.y0 + cases.random_state(case.mesh, case.N, seed=seed)
    y[case.dirichlet_mask, 0:3] = case.y0[case.dirichlet_mask, 0:3]
    y[:, :, 0, 1] = 0.0
    return y


@pytest.mark.parametrize("N", [3, 7])
def test_noalloc_residual_matches_allocating_residual_twice(N):
    import torch
    import paper_2311_09465_gb300 as ts
    case = cases.junction_case(N=N, Re=300.0, Wo=8.0, mesh=mg.junction(h=0.6, seed=3))
    g = ts.GLSProblem(case)
    for call, seed in enumerate((1, 2)):          # two calls in a row, different states
        y = to_dev(_state(case, seed), torch.float32)
        ref = to_np(ts.ts_residual(g.prob, y, g.field(torch.float32)))
        r = torch.full_like(y, float("nan"))       # the entry point must overwrite r
        ts.ts_residual_noalloc(g.prob, y, r)
        torch.cuda.synchronize()
        got = to_np(r)
        assert np.all(np.isfinite(got)), call
        assert rel_l2(got, ref) <= 1e-5, (call, rel_l2(got, ref))
    g.close()


def test_noalloc_residual_rejects_meshes_beyond_its_scratch():
    import torch
    import paper_2311_09465_gb300 as ts
    mesh = mg.junction(h=0.25, seed=1)              # about 22k tets: needs > 32 MiB at N = 7
    case = cases.junction_case(N=7, Re=300.0, Wo=8.0, mesh=mesh)
    g = ts.GLSProblem(case)
    y = g.field(torch.float32)
    with pytest.raises(ts.TsError) as ei:
        ts.ts_residual_noalloc(g.prob, y, g.field(torch.float32))
    assert ei.value.code == ts.TS_ERR_ARG and "scratch" in str(ei.value)
    g.close()
