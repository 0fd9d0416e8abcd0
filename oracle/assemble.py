"""Dense tangent matrix H built block by block from eq. (K_mat), section 2.4.

For small meshes only.  Written from the block formulas, not from the
operator code, so that it pins the Jacobian-vector products:

  K_AB   = int [rho N_A Omega N_B + rho N_A A_k dN_B/dx_k + mu dN_A/dx_k dN_B/dx_k I]
         + int (-Omega N_A + A_k dN_A/dx_k) rho tau (Omega N_B + A_k dN_B/dx_k)
  G_AB,i = -int dN_A/dx_i N_B I + int (-Omega N_A + A_k dN_A/dx_k) tau dN_B/dx_i
  D_AB,j =  int N_A dN_B/dx_j I + int dN_A/dx_j tau (Omega N_B + A_k dN_B/dx_k)
  L_AB   =  int (1/rho) dN_A/dx_k tau dN_B/dx_k

H = [[K,0,0,G1],[0,K,0,G2],[0,0,K,G3],[D1,D2,D3,L]] (eq. tangent).  Variant
'paper' drops the least-squares parts of G and D (section 2.5.2).  The
pseudo-time mass (N_A, c1 rho/dt N_B I) is added to K (section 2.5.3) and a
resistance outlet adds R (int N_A n_i)(int N_B n_j) per mode.

The complex blocks act on conjugate-symmetric mode vectors; ``to_real``
writes them in the real unknowns of section 2.5.1 (re/im of modes
0..N-1 per field), the layout of the operator functions.
"""
from __future__ import annotations

import numpy as np

from .geometry import QP_BARY, face_normals_areas
from .operator import Linearization, Problem
from .spectral import omega_diag


def dense_tangent_complex(prob: Problem, lin: Linearization, variant: str = "frozen",
                          mass_coef: float = 0.0) -> np.ndarray:
    """Complex H indexed [A, field, m, B, field, n] (modes -N+1..N-1)."""
    V, nm, rho, mu = prob.n_nodes, prob.nm, prob.rho, prob.mu
    H = np.zeros((V, 4, nm, V, 4, nm), dtype=np.complex128)
    Om = np.diag(omega_diag(prob.N, prob.omega))
    I = np.eye(nm)
    for ie, e in enumerate(lin.elems):
        t = prob.tets[e]
        dN = prob.dN[e]
        vol = prob.vol[e]
        for q in range(4):
            lam = QP_BARY[q]
            w = vol / 4.0
            Ak = lin.A[ie, q]
            tau = lin.tau[ie, q]
            for a in range(4):
                adv_a = sum(Ak[k] * dN[a, k] for k in range(3))
                test_a = -Om * lam[a] + adv_a
                for b in range(4):
                    adv_b = sum(Ak[k] * dN[b, k] for k in range(3))
                    trial_b = Om * lam[b] + adv_b
                    Kab = w * (rho * lam[a] * Om * lam[b] + rho * lam[a] * adv_b) \
                        + w * rho * test_a @ tau @ trial_b
                    Lab = w / rho * (dN[a] @ dN[b]) * tau
                    for i in range(3):
                        H[t[a], i, :, t[b], i, :] += Kab
                        Gi = -w * dN[a, i] * lam[b] * I
                        Dj = w * lam[a] * dN[b, i] * I
                        if variant == "frozen":
                            Gi = Gi + w * test_a @ tau * dN[b, i]
                            Dj = Dj + w * dN[a, i] * tau @ trial_b
                        H[t[a], i, :, t[b], 3, :] += Gi
                        H[t[a], 3, :, t[b], i, :] += Dj
                    H[t[a], 3, :, t[b], 3, :] += Lab
        for a in range(4):
            for b in range(4):
                visc = mu * vol * (dN[a] @ dN[b]) * I
                mass = mass_coef * vol / 20.0 * (2.0 if a == b else 1.0) * I
                for i in range(3):
                    H[t[a], i, :, t[b], i, :] += visc + mass
    for faces, R in prob.outlets:
        n, area = face_normals_areas(prob.xyz, faces)
        wn = np.zeros((V, 3))
        np.add.at(wn, faces, np.repeat(((area / 3.0)[:, None] * n)[:, None, :], 3, axis=1))
        for i in range(3):
            for j in range(3):
                outer = R * np.outer(wn[:, i], wn[:, j])
                H[:, i, :, :, j, :] += outer[:, None, :, None] * I[None, :, None, :]
    return H


def to_real(Hc: np.ndarray, prob: Problem) -> np.ndarray:
    """Real matrix on the storage layout [V,4,N,2] x [V,4,N,2], with fixed rows/columns zero."""
    V, N, nm = prob.n_nodes, prob.N, prob.nm
    # unit complex inputs for each real unknown (n, re/im)
    X = np.zeros((nm, N, 2), dtype=np.complex128)
    X[N - 1, 0, 0] = 1.0
    for n in range(1, N):
        X[N - 1 + n, n, 0] = 1.0
        X[N - 1 - n, n, 0] = 1.0
        X[N - 1 + n, n, 1] = 1j
        X[N - 1 - n, n, 1] = -1j
    X = X.reshape(nm, 2 * N)
    Y = np.einsum("afmbgn,nk->afmbgk", Hc, X)             # inputs -> real columns
    Yp = Y[:, :, N - 1:]                                    # outputs m = 0..N-1
    Hr = np.stack([Yp.real, Yp.imag], axis=3)              # [V,4,N,2,V,4,2N]
    Hr = Hr.reshape(V, 4, N, 2, V, 4, N, 2)
    Hr[:, :, 0, 1] = 0.0
    Hr[prob.dmask, 0:3] = 0.0
    Hr[:, :, :, :, prob.dmask, 0:3] = 0.0
    return Hr.reshape(V * 4 * N * 2, V * 4 * N * 2)
