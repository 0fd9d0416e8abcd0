"""Linear and nonlinear solvers of sections 2.4-2.5 (FP64, plain).

* ``gmres``: restarted GMRES (Saad & Schultz 1986, cited by the paper for
  its linear solver) with modified Gram-Schmidt and Givens rotations; the
  stopping rule is ||b - A x|| <= tol ||b|| (tolerance epsilon_LS of
  section 2.4 remark 6, relative to the initial linear residual with x0 = 0).
* ``dense_solve``: LU of the dense tangent restricted to the free unknowns.
* ``pseudo_time_solve``: one Newton step per pseudo-time step (section
  2.5.3): (H + c1 rho / dt M) delta = -r, y <- y + delta on free unknowns,
  Dirichlet values kept as initialised (section 2.4 remarks 1-2), stop when
  ||r|| <= tol * r_ref.  dt = inf is plain Newton-Raphson, eq. (NR).

Pinned by: tests/test_oracle_solver.py (GMRES equals dense LU; the
pseudo-time and Newton paths reach the same root; the root has a residual
below the tolerance when re-evaluated).
"""
from __future__ import annotations

import math

import numpy as np

from . import operator as op
from .assemble import dense_tangent_complex, to_real


def gmres(matvec, b, tol=0.05, m=100, maxiter=10000):
    """Solve A x = b from x0 = 0.  Returns (x, n_matvec, history of ||r||/||b||)."""
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    nmv = 0
    r = b.copy()
    while nmv < maxiter:
        beta = np.linalg.norm(r)
        Vb = np.zeros((m + 1, n))
        Hh = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Vb[0] = r / beta
        k_used = 0
        for k in range(m):
            w = matvec(Vb[k])
            nmv += 1
            for j in range(k + 1):
                Hh[j, k] = Vb[j] @ w
                w = w - Hh[j, k] * Vb[j]
            Hh[k + 1, k] = np.linalg.norm(w)
            if Hh[k + 1, k] > 0:
                Vb[k + 1] = w / Hh[k + 1, k]
            for j in range(k):
                t = cs[j] * Hh[j, k] + sn[j] * Hh[j + 1, k]
                Hh[j + 1, k] = -sn[j] * Hh[j, k] + cs[j] * Hh[j + 1, k]
                Hh[j, k] = t
            d = math.hypot(Hh[k, k], Hh[k + 1, k])
            cs[k], sn[k] = Hh[k, k] / d, Hh[k + 1, k] / d
            Hh[k, k] = d
            Hh[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) <= tol * bnorm or nmv >= maxiter:
                break
        yk = np.linalg.solve(np.triu(Hh[:k_used, :k_used]), g[:k_used])
        x = x + Vb[:k_used].T @ yk
        r = b - matvec(x)
        nmv += 1
        if np.linalg.norm(r) <= tol * bnorm * (1 + 1e-12):
            break
    return x, nmv, hist


def dense_matrix(prob: op.Problem, lin: op.Linearization, variant="paper", mass_coef=0.0):
    return to_real(dense_tangent_complex(prob, lin, variant, mass_coef), prob)


def dense_solve(Hr: np.ndarray, b: np.ndarray, free: np.ndarray) -> np.ndarray:
    x = np.zeros(b.size)
    idx = np.nonzero(free.ravel())[0]
    x[idx] = np.linalg.solve(Hr[np.ix_(idx, idx)], b[idx])
    return x


def pseudo_time_solve(prob: op.Problem, y0: np.ndarray, dt: float = math.inf, tol: float = 1e-8,
                      r_ref: float | None = None, max_steps: int = 200, linear: str = "gmres",
                      eps_ls: float = 0.05, krylov: int = 100, c1: float = 1.5,
                      variant: str = "paper", max_matvec: int = 10000, verbose: bool = False):
    """Return (y, report).  ``linear`` is 'gmres' or 'dense'."""
    y = y0.copy()
    free = op.free_mask(prob)
    mass = 0.0 if math.isinf(dt) else c1 * prob.rho / dt
    hist = []
    nmv_total = 0
    for step in range(max_steps + 1):
        lin = op.linearize(prob, y)
        r = op.apply(prob, lin, y, "frozen")
        rn = float(np.linalg.norm(r))
        if r_ref is None:
            r_ref = rn
        hist.append(rn / r_ref)
        if verbose:
            print(f"step {step}: |r|/r_ref = {rn / r_ref:.3e}")
        if rn <= tol * r_ref or step == max_steps:
            break
        b = -r.ravel()
        if linear == "dense":
            Hr = dense_matrix(prob, lin, variant, mass)
            dy = dense_solve(Hr, b, free)
        else:
            def mv(v):
                return op.jvp(prob, lin, v.reshape(y.shape), variant, mass).ravel()
            dy, nmv, _ = gmres(mv, b, tol=eps_ls, m=krylov, maxiter=max_matvec)
            nmv_total += nmv
        y = y + np.where(free, dy.reshape(y.shape), 0.0)
    return y, dict(steps=step, hist=hist, r_ref=r_ref, matvecs=nmv_total,
                   converged=hist[-1] <= tol)
