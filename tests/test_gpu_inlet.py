"""Inflow boundary data inside the library (ts_set_inlet, ts_initial_guess).

The library turns flow-rate coefficients Q_n into Dirichlet velocity modes
at the inlet nodes (section 2.4, eq. upgh_def; parabolic profile of section
3.1, or the Womersley mode profiles of fully developed pulsatile pipe flow).
Checks:
* pipe (wall exactly at r = R): the derived centre, axis and radius are the
  pipe's; every inlet value equals the oracle's Womersley closed form
  (``oracle.womersley``, its own Bessel series) and the seeded input
  generator's (scipy's Bessel functions) to 1e-12; all other entries zero;
* junction: the parabolic values equal the closed form on the derived
  geometry, that geometry is the arm's, and the discrete flow rate through
  the inlet triangles approaches Q_n;
* the FP32 initial guess is the FP64 one rounded.
"""
import numpy as np
import pytest

from oracle import womersley as wo
from workloads import cases, meshgen as mg

from gpu_util import to_np

pytestmark = pytest.mark.gpu


def test_pipe_womersley_inlet_matches_closed_form():
    import torch
    import paper_2311_09465_gb300 as ts
    case = cases.pipe_case(N=3, Re=100.0, Wo=5.0, amps=(1.0, 0.5 + 0.2j, 0.25 - 0.1j),
                           mesh=mg.pipe(nc=4, nr=4, nz=20))
    R = case.info["R"]
    U = np.asarray(case.info["U"])
    g = ts.GLSProblem(case)
    g.set_inlet(mg.TAG_INLET1, U * np.pi * R ** 2, "womersley")
    info = g.inlet_info(mg.TAG_INLET1)
    assert abs(info["radius"] - R) <= 1e-9 * R
    np.testing.assert_allclose(info["centre"], [0.0, 0.0, 0.0], atol=1e-9)
    np.testing.assert_allclose(info["direction"], [0.0, 0.0, 1.0], atol=1e-12)
    y = to_np(g.initial_guess(torch.float64))
    wall = cases.nodes_with_tag(case.mesh, mg.TAG_WALL)
    inlet = cases.nodes_with_tag(case.mesh, mg.TAG_INLET1) & ~wall
    r = np.hypot(case.mesh.xyz[inlet, 0], case.mesh.xyz[inlet, 1])
    ref = np.zeros_like(y)
    for n in range(case.N):
        w = wo.mode_profile(r, R, U[n], n, case.omega, case.mu / case.rho)
        ref[inlet, 2, n, 0] = np.real(w)
        ref[inlet, 2, n, 1] = 0.0 if n == 0 else np.imag(w)
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 1e-12 * scale
    # the seeded generator (scipy's complex Bessel functions) gives the same data
    assert np.abs(y - case.y0).max() <= 1e-12 * scale
    y32 = to_np(g.initial_guess(torch.float32))
    assert np.abs(y32 - y.astype(np.float32)).max() == 0.0
    g.close()


def test_junction_parabolic_inlets_closed_form_and_flow_rate():
    import torch
    import paper_2311_09465_gb300 as ts
    case = cases.junction_case(N=4, Re=300.0, Wo=8.0, mesh=mg.junction(h=0.3, seed=3))
    g = ts.GLSProblem(case)
    arms = {tag: (ax, sg, R) for ax, sg, R, tag in mg.JUNCTION_ARMS}
    Qs = {}
    for tag in (mg.TAG_INLET1, mg.TAG_INLET2):
        R = arms[tag][2]
        Qs[tag] = np.asarray(case.info["waves"][tag]) * np.pi * R ** 2
        g.set_inlet(tag, Qs[tag], "parabolic")
    y = to_np(g.initial_guess(torch.float64))
    xyz = case.mesh.xyz
    touched = np.zeros(case.mesh.n_nodes, dtype=bool)
    for tag in (mg.TAG_INLET1, mg.TAG_INLET2):
        ax, sg, R = arms[tag]
        info = g.inlet_info(tag)
        ai = mg._AX[ax]
        # geometry of the arm: inflow along -sg * axis, centre on the axis, radius close to R
        d_ref = np.zeros(3)
        d_ref[ai] = -sg
        np.testing.assert_allclose(info["direction"], d_ref, atol=1e-6)
        off = info["centre"].copy()
        off[ai] = 0.0
        assert np.linalg.norm(off) <= 0.05 * R
        assert abs(info["radius"] - R) <= 0.05 * R
        # values: the parabola on the derived geometry, along the derived direction
        faces = case.mesh.bfaces[case.mesh.btag == tag]
        nodes = np.unique(faces)
        others = np.unique(case.mesh.bfaces[case.mesh.btag != tag])
        rim = np.isin(nodes, others)
        Rf, c, d = info["radius"], info["centre"], info["direction"]
        rel = xyz[nodes] - c
        rperp = np.linalg.norm(rel - np.outer(rel @ d, d), axis=1)
        for n in range(case.N):
            U = Qs[tag][n] / (np.pi * Rf ** 2)
            w = 2.0 * U * (1.0 - np.minimum(rperp / Rf, 1.0) ** 2)
            w[rim] = 0.0
            for i in range(3):
                np.testing.assert_allclose(y[nodes, i, n, 0], np.real(w) * d[i], rtol=0,
                                           atol=1e-12 * abs(U) * 2)
                im = 0.0 if n == 0 else np.imag(w) * d[i]
                np.testing.assert_allclose(y[nodes, i, n, 1], im, rtol=0, atol=1e-12 * abs(U) * 2)
        # discrete flow rate of mode 0 through the inlet triangles (P1 interpolation)
        a, b, cc = xyz[faces[:, 0]], xyz[faces[:, 1]], xyz[faces[:, 2]]
        nrm = np.cross(b - a, cc - a) / 2.0           # outward, area-weighted
        un = np.einsum("fki,fi->fk", y[faces, 0:3, 0, 0], -nrm)
        q0 = un.sum(axis=1).sum() / 3.0
        assert abs(q0 - Qs[tag][0].real) <= 0.08 * abs(Qs[tag][0].real), (q0, Qs[tag][0])
        touched[nodes] = True
    # nothing outside the inlets, pressure zero
    assert np.abs(y[~touched]).max() == 0.0
    assert np.abs(y[:, 3]).max() == 0.0
    g.close()
