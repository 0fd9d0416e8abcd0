"""Writes junction_re300_N3.npz: the oracle's converged field on a small junction.

The Fontan-like cross junction of the configurations at a coarse mesh
(``meshgen.junction(h=0.7, seed=3)``: 461 nodes, 1205 tetrahedra), N = 3,
Re 300, Wo 8, random 1/n^2 inflow waveforms (amplitude 0.2, seeds 100 and
101), resistance outlets R = 1.  The root of the oracle's residual (eq. Rmc)
is found by pseudo-time Newton steps (section 2.5.3) whose linear solves are
GMRES on the oracle's LIN_A tangent products, right-preconditioned by an LU
factorisation of the oracle's dense frozen tangent (eq. K_mat), solved to
1e-8 so every step is a Newton step of the tau-frozen derivative.  Only the
oracle's residual, tangent products and dense assembly enter; the path does
not change the root, which is checked at the end: ||r(y)|| <= 1e-11 r_ref
with r_ref = ||r(y0)|| of the paper's initial guess (section 2.4).

Run from the repository root: python tests/golden/make_junction_re300.py
"""
import math
import os
import sys

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import operator as op  # noqa: E402
from oracle import solver as sv  # noqa: E402
from workloads import cases, meshgen as mg  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "junction_re300_N3.npz")


def case():
    return cases.junction_case(N=3, Re=300.0, Wo=8.0, wave_seed=100, resistance=1.0,
                               mesh=mg.junction(h=0.7, seed=3), amp=0.2)


def main():
    c = case()
    prob = op.problem_from_case(c)
    free = op.free_mask(prob)
    idx = np.nonzero(free.ravel())[0]
    y = c.y0.copy()
    r_ref = float(np.linalg.norm(op.residual(prob, y)))
    dt0, hist = 0.5, []
    for step in range(60):
        lin = op.linearize(prob, y)
        r = op.apply(prob, lin, y, "frozen")
        rn = float(np.linalg.norm(r))
        hist.append(rn / r_ref)
        print(f"step {step}: |r|/r_ref = {rn / r_ref:.3e}", flush=True)
        if rn <= 1e-12 * r_ref:
            break
        # switched evolution relaxation of the pseudo-time step
        dt = dt0 * (r_ref / rn)
        mass = 0.0 if dt > 1e6 else c.c1 * c.rho / dt
        P = sv.dense_matrix(prob, lin, "frozen", mass)
        lu = sla.lu_factor(P[np.ix_(idx, idx)])

        def pinv(v):
            x = np.zeros(v.size)
            x[idx] = sla.lu_solve(lu, v[idx])
            return x

        def mv(u):
            return op.jvp(prob, lin, pinv(u).reshape(y.shape), "lin_a", mass).ravel()

        u, _, _ = sv.gmres(mv, -r.ravel(), tol=1e-8, m=100, maxiter=2000)
        y = y + np.where(free, pinv(u).reshape(y.shape), 0.0)
    final = float(np.linalg.norm(op.residual(prob, y)))
    assert final <= 1e-11 * r_ref, final / r_ref
    np.savez_compressed(OUT, y=y, r_ref=r_ref, hist=np.array(hist),
                        n_nodes=c.mesh.n_nodes, n_tets=c.mesh.n_tets)
    print("wrote", OUT, "final", final / r_ref)


if __name__ == "__main__":
    main()
