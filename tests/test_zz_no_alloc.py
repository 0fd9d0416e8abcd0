"""The allocation-free residual entry point (ts_residual_noalloc).

It serves callers that cannot allocate device memory at call time; it must
give the same residual as ts_residual in FP32, on repeated calls that reuse
its fixed scratch array, and refuse meshes too large for that array.  This
file is collected last so that a failure here stops a -x run only after all
other tests have run.
"""
import os
import subprocess
import sys
import textwrap

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


_FRESH_PROCESS = textwrap.dedent("""
    import sys
    import torch
    import paper_2311_09465_gb300 as ts
    from workloads import cases, meshgen as mg
    torch.cuda.set_device(0)
    case = cases.junction_case(N=7, Re=300.0, Wo=8.0, mesh=mg.junction(h=0.6, seed=3))
    g = ts.GLSProblem(case)                        # set-up: may allocate
    y = torch.tensor(case.y0, dtype=torch.float32, device="cuda")
    r = torch.empty_like(y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):                             # the first call on this device, then another
        ts.ts_residual_noalloc(g.prob, y, r)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.isfinite(r).all()
    print("FREE", free0, free1)
    sys.exit(0 if free1 >= free0 else 3)
""")


def test_noalloc_first_call_in_fresh_process_allocates_no_device_memory():
    # in a process of its own, so that nothing earlier has loaded the library's
    # kernels or arrays: the set-up (problem creation) does that, the calls not
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    env.pop("CUDA_MODULE_LOADING", None)            # CUDA's default: lazy loading
    out = subprocess.run([sys.executable, "-c", _FRESH_PROCESS], cwd=root, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
