"""Steady SUPG/PSPG residual of the time formulation, App. B eq. (NSt-weak).

Written independently of ``operator.py`` (real scalar arithmetic, scalar
tau, no mode matrices) to pin the time-spectral residual in its steady
limit: the paper states (App. B) that eq. (NS-weak) reduces to eq.
(NSt-weak) for linear shape functions when omega = 0 and the flow is
steady.  tau is eq. (3D-taut) with omega_hat = 0:

  tau = [u_i G_ij u_j + C_I kappa^2 G_ij G_ij]^{-1/2}.

Momentum (steady, second derivatives dropped):
  r_i = rho u_j du_i/dx_j + dp/dx_i
  R^m_{ai} = int rho N_a u_j du_i/dx_j - dN_a/dx_i p + mu dN_a/dx_j du_i/dx_j
           + int (u_j dN_a/dx_j) tau r_i                       (SUPG)
  R^c_a    = int N_a du_i/dx_i + int (1/rho) dN_a/dx_i tau r_i  (PSPG)

Parity: this function is itself the pin for the spectral residual's
mode-0 limit.  It is pinned on its own by closed forms per element in
tests/test_oracle_steady.py, assembled with independently computed geometry:
the u = 0 Stokes limit (pressure and PSPG terms), uniform flow with a linear
pressure (SUPG and PSPG with a constant tau), and the Galerkin terms with the
stabilisation switched off (exact P1 mass matrix, stiffness, divergence).
"""
from __future__ import annotations

import numpy as np

from .geometry import QP_BARY, tet_geometry


def steady_residual(xyz, tets, u, p, rho, mu, C_I, dmask):
    """Return (R^m [V,3], R^c [V]) for real nodal fields u [V,3], p [V]."""
    dN, vol, G = tet_geometry(xyz, tets)
    nu = mu / rho
    V = xyz.shape[0]
    Rm = np.zeros((V, 3))
    Rc = np.zeros(V)
    GG = np.einsum("eij,eij->e", G, G)
    for e in range(tets.shape[0]):
        t = tets[e]
        ua = u[t]                    # [4,3]
        pa = p[t]                    # [4]
        gu = dN[e].T @ ua            # gu[j, i] = du_i/dx_j
        gp = dN[e].T @ pa            # [3]
        div = np.trace(gu)
        w = vol[e] / 4.0
        for q in range(4):
            lam = QP_BARY[q]
            uq = lam @ ua
            pq = lam @ pa
            tau = (uq @ G[e] @ uq + C_I * nu * nu * GG[e]) ** -0.5
            adv = uq @ gu            # u_j du_i/dx_j, [3]
            r = rho * adv + gp
            supg = dN[e] @ uq        # u_j dN_a/dx_j, [4]
            for a in range(4):
                Rm[t[a]] += w * (rho * lam[a] * adv - dN[e, a] * pq + supg[a] * tau * r)
                Rc[t[a]] += w * (lam[a] * div + (1.0 / rho) * tau * (dN[e, a] @ r))
        for a in range(4):
            Rm[t[a]] += mu * vol[e] * (gu.T @ dN[e, a])
    Rm[dmask] = 0.0
    return Rm, Rc
