"""Tracer residual of eq. (3D-weak) on the GPU (ts_tracer_residual) vs the oracle.

Bars: relative L2 <= 1e-12 in FP64 and <= 1e-5 in FP32 against
``oracle.tracer.tracer_residual`` on the same seeded velocity and scalar
fields (pipes and a junction, N = 1 ... 15, several tiles and a ragged
tail); Dirichlet rows and Im(mode 0) exactly zero; the residual is linear in
phi (it is its own tangent).
"""
import numpy as np
import pytest

from oracle import tracer as tr
from workloads import cases, meshgen as mg

from gpu_util import rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}

MESHES = {
    "pipe_N1": (lambda: mg.pipe(nc=2, nr=1, nz=3, seed=7), 1),
    "pipe_N4": (lambda: mg.pipe(nc=2, nr=2, nz=4, seed=7), 4),
    "junction_N3": (lambda: mg.junction(h=0.6, seed=3), 3),
    "pipe_N7": (lambda: mg.pipe(nc=3, nr=2, nz=5, seed=2), 7),
    "pipe_N15": (lambda: mg.pipe(nc=2, nr=1, nz=2, seed=7), 15),
}


def _modes(rng, shape, N, scale=1.0):
    x = scale * rng.standard_normal(shape + (N, 2))
    x *= (1.0 / (1.0 + np.arange(N)) ** 2)[:, None]
    x[..., 0, 1] = 0.0
    return x


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", list(MESHES))
def test_tracer_residual_matches_oracle(name, prec):
    import torch
    import paper_2311_09465_gb300 as ts
    make, N = MESHES[name]
    mesh = make()
    rng = np.random.default_rng(21)
    kappa, omega = 0.03, 0.8
    a = _modes(rng, (mesh.n_nodes, 3), N, 2.0)
    phi = _modes(rng, (mesh.n_nodes,), N)
    dmask = cases.dirichlet_nodes(mesh, (mg.TAG_INLET1,))
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, N, kappa, omega, dmask, 3.0)
    ref = tr.tracer_residual(tp, a, phi)
    m = ts.ts_mesh_load(mesh.xyz, mesh.tets, mesh.bfaces, mesh.btag)
    t = ts.Tracer(m, mesh.n_nodes, N, kappa, omega, 3.0, dirichlet_tags=(mg.TAG_INLET1,))
    dty = torch.float64 if prec == 64 else torch.float32
    got = to_np(t.residual(to_dev(a, dty), to_dev(phi, dty)))
    assert rel_l2(got, ref) <= TOL[prec], rel_l2(got, ref)
    assert np.all(got[:, 0, 1] == 0)
    assert np.all(got[dmask] == 0)
    if prec == 64:
        # linear in phi: r(phi1 + 2 phi2) = r(phi1) + 2 r(phi2)
        phi2 = _modes(rng, (mesh.n_nodes,), N)
        r1 = to_np(t.residual(to_dev(a, dty), to_dev(phi, dty)))
        r2 = to_np(t.residual(to_dev(a, dty), to_dev(phi2, dty)))
        r12 = to_np(t.residual(to_dev(a, dty), to_dev(phi + 2 * phi2, dty)))
        assert rel_l2(r12, r1 + 2 * r2) <= 1e-13
    t.close()
    ts.ts_mesh_free(m)


def test_tracer_solve_reaches_the_oracle_root_and_gls_bounds_the_step():
    # a step of tracer entering a pipe with a pulsating axial velocity at a cell
    # Peclet number near 50: the GLS solution is the root of the oracle's
    # residual, every mode is energised by the coupling (section 3.3), and it
    # stays near [0, 1] where the Galerkin-only method over- and undershoots
    import torch
    import paper_2311_09465_gb300 as ts
    mesh = mg.pipe(nc=3, nr=2, nz=12, seed=4)
    N, kappa, omega = 4, 0.004, 1.2
    V = mesh.n_nodes
    a = np.zeros((V, 3, N, 2))
    a[:, 2, 0, 0] = 1.0
    a[:, 2, 1, 0] = 0.3
    inlet = cases.nodes_with_tag(mesh, mg.TAG_INLET1)
    phi0 = np.zeros((V, N, 2))
    phi0[inlet & (mesh.xyz[:, 0] > 0), 0, 0] = 1.0
    m = ts.ts_mesh_load(mesh.xyz, mesh.tets, mesh.bfaces, mesh.btag)
    out = {}
    for gls in (True, False):
        t = ts.Tracer(m, V, N, kappa, omega, 3.0, dirichlet_tags=(mg.TAG_INLET1,))
        t.stabilised(gls)
        phi = to_dev(phi0, torch.float64)
        rep = t.solve(to_dev(a, torch.float64), phi, tol=1e-10, krylov=100, max_matvec=20000)
        assert rep["rel"] <= 1e-10, rep
        out[gls] = to_np(phi)
        t.close()
    ts.ts_mesh_free(m)
    tp = tr.make_tracer_problem(mesh.xyz, mesh.tets, N, kappa, omega, inlet, 3.0)
    r0 = np.linalg.norm(tr.tracer_residual(tp, a, phi0))
    assert np.linalg.norm(tr.tracer_residual(tp, a, out[True])) <= 1e-8 * r0
    # the inlet data stay, Im(mode 0) stays zero, the pulsation energises the higher modes
    np.testing.assert_array_equal(out[True][inlet], phi0[inlet])
    assert np.all(out[True][:, 0, 1] == 0)
    assert np.abs(out[True][:, 1:]).max() > 1e-3
    # boundedness of the mean (mode 0) field: GLS near [0, 1], Galerkin worse
    over = {g: max(out[g][:, 0, 0].max() - 1.0, -out[g][:, 0, 0].min()) for g in out}
    assert over[True] < 0.15, over
    assert over[False] > over[True], over
