"""Inflow boundary data inside the library (ts_set_inlet, ts_initial_guess).

The library turns flow-rate coefficients Q_n into Dirichlet velocity modes
at the inlet nodes (section 2.4, eq. upgh_def; parabolic profile of section
3.1, or the Womersley mode profiles of fully developed pulsatile pipe flow).
Checks:
* pipe (wall exactly at r = R): the derived centre, axis and radius are the
  pipe's; every inlet value equals the oracle's Womersley closed form
  (``oracle.womersley``, its own Bessel series) and the seeded input
  generator's (scipy's Bessel functions) to 1e-12; all other entries zero;
  the discrete flow rate through the inlet triangles approaches Q_n;
* junction (inlet caps carved from a lattice, arm geometry given): the
  parabolic values equal the closed form and the generator's data;
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
    # the discrete flow rate through the inlet triangles (P1 interpolation of
    # the profile on the polygonal disk) approaches Q_n = pi R^2 U_n
    xyz = case.mesh.xyz
    faces = case.mesh.bfaces[case.mesh.btag == mg.TAG_INLET1]
    a, b, cc = xyz[faces[:, 0]], xyz[faces[:, 1]], xyz[faces[:, 2]]
    nrm = np.cross(b - a, cc - a) / 2.0                # outward, area-weighted
    for n in range(case.N):
        q = sum(np.einsum("fki,fi->", y[faces, 0:3, n, part], -nrm) / 3.0 * (1j if part else 1)
                for part in (0, 1))
        assert abs(q - np.pi * R ** 2 * U[n]) <= 0.06 * abs(np.pi * R ** 2 * U[n]), (n, q)
    y32 = to_np(g.initial_guess(torch.float32))
    assert np.abs(y32 - y.astype(np.float32)).max() == 0.0
    g.close()


def test_junction_parabolic_inlets_closed_form_and_flow_rate():
    import torch
    import paper_2311_09465_gb300 as ts
    case = cases.junction_case(N=4, Re=300.0, Wo=8.0, mesh=mg.junction(h=0.3, seed=3))
    g = ts.GLSProblem(case)
    Qs = {}
    for ax, sg, R, tag in mg.JUNCTION_ARMS:
        if tag not in (mg.TAG_INLET1, mg.TAG_INLET2):
            continue
        ai = mg._AX[ax]
        # the mesh's inlet caps are carved from a lattice: the arm's geometry is given
        d = np.zeros(3)
        d[ai] = -sg
        c = np.zeros(3)
        c[ai] = sg * 6.0
        Qs[tag] = np.asarray(case.info["waves"][tag]) * np.pi * R ** 2
        g.set_inlet(tag, Qs[tag], "parabolic", centre=c, direction=d, radius=R)
        info = g.inlet_info(tag)
        np.testing.assert_allclose(info["direction"], d, atol=0)
        assert info["radius"] == R
    y = to_np(g.initial_guess(torch.float64))
    xyz = case.mesh.xyz
    # the parabola 2 U_n (1 - r^2/R^2), U_n = Q_n / (pi R^2), cut at the wall
    ref = np.zeros_like(y)
    wall = cases.nodes_with_tag(case.mesh, mg.TAG_WALL)
    for ax, sg, R, tag in mg.JUNCTION_ARMS:
        if tag not in Qs:
            continue
        ai = mg._AX[ax]
        o = [k for k in range(3) if k != ai]
        nodes = np.nonzero(cases.nodes_with_tag(case.mesh, tag) & ~wall)[0]
        r = np.hypot(xyz[nodes, o[0]], xyz[nodes, o[1]])
        for n in range(case.N):
            w = 2.0 * Qs[tag][n] / (np.pi * R ** 2) * (1.0 - np.minimum(r / R, 1.0) ** 2)
            ref[nodes, ai, n, 0] = -sg * np.real(w)
            ref[nodes, ai, n, 1] = 0.0 if n == 0 else -sg * np.imag(w)
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 1e-12 * scale
    # the seeded generator builds the same Dirichlet data
    assert np.abs(y - case.y0).max() <= 1e-12 * scale
    # derived geometry: the cap's normal is the arm's axis
    g.set_inlet(mg.TAG_INLET1, Qs[mg.TAG_INLET1], "parabolic")
    np.testing.assert_allclose(g.inlet_info(mg.TAG_INLET1)["direction"], [0.0, -1.0, 0.0], atol=1e-9)
    g.close()
