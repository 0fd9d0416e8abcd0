"""Time-spectral GLS convection-diffusion of a scalar (a passive tracer),
eq. (3D-weak) with the residual of eq. (3D-weak-def), section 2.2.

Test infrastructure only: plain FP64 numpy, written from the paper, sharing
no code with the CUDA path.

Unknown: a scalar phi with N independent modes at the mesh nodes (storage
[V][N][2], the layout of one field of the flow solver).  Given: the
advecting velocity a_i (modes at the nodes, [V][3][N][2]; A_i = A(a_i) at
each quadrature point, eq. phi-def), the diffusivity kappa, the base
frequency omega, Dirichlet data on Gamma_g (rows of those nodes are not
equations) and zero Neumann data elsewhere.

For every element and quadrature point (weights V/4, N_A barycentric):

  res   = Omega phi + A_i dphi/dx_i      strong residual; kappa's second
                                         derivative vanishes on P1 elements
  T     = tau res                        tau of eq. (3D-tau) with kappa
  r_A  += w N_A res                      Galerkin: (w, Omega phi + A_i dphi/dx_i)
        + w kappa dN_A/dx_i dphi/dx_i    (dw/dx_i, kappa dphi/dx_i)
        + w [(-Omega N_A) T + dN_A/dx_i A_i T]
                                         (res(w), tau res(phi)): for w = N_A e_m,
                                         res(w)^H = e_m^T (Omega^H N_A + dN_A/dx_i A_i^H)
                                         with Omega^H = -Omega, A_i Hermitian

The residual is linear in phi for a given velocity, so it is also its own
tangent.

Pinned by: tests/test_oracle_tracer.py -- the one-mode case equals an
independently written steady SUPG/GLS residual with the scalar tau; the
velocity-free one-mode case equals kappa times the P1 stiffness matrix;
conjugate symmetry of the complex rows and Im r_0 = 0; interior rows vanish
for a linear field orthogonal to a uniform time-periodic velocity; and the
energy identity Re(phi^H r(phi)) = kappa |grad phi|^2 + |tau^{1/2} res|^2 for a
uniform velocity and phi = 0 on the boundary (the Galerkin convective and
Omega terms carry no real part there).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .geometry import QP_BARY, tet_geometry
from .spectral import conv_matrix, omega_diag, to_complex, to_storage
from .tau import tau_matrix


@dataclass
class TracerProblem:
    xyz: np.ndarray
    tets: np.ndarray
    N: int
    kappa: float
    omega: float
    C_I: float
    dmask: np.ndarray      # [V] bool: Dirichlet nodes (no equation there)
    dN: np.ndarray = None
    vol: np.ndarray = None
    G: np.ndarray = None

    @property
    def nm(self) -> int:
        return 2 * self.N - 1


def make_tracer_problem(xyz, tets, N, kappa, omega, dmask, C_I=3.0) -> TracerProblem:
    dN, vol, G = tet_geometry(np.asarray(xyz, np.float64), np.asarray(tets))
    return TracerProblem(xyz=np.asarray(xyz, np.float64), tets=np.asarray(tets, np.int64), N=N,
                         kappa=float(kappa), omega=float(omega), C_I=float(C_I),
                         dmask=np.asarray(dmask, bool), dN=dN, vol=vol, G=G)


def tracer_residual(tp: TracerProblem, a: np.ndarray, phi: np.ndarray, return_complex: bool = False,
                    chunk: int = 2048) -> np.ndarray:
    """Residual of eq. (3D-weak) for the tracer phi [V][N][2] advected by a [V][3][N][2]."""
    N, nm = tp.N, tp.nm
    Phi = to_complex(phi, N)                               # [V, nm]
    Av = to_complex(a, N)                                  # [V, 3, nm]
    om = omega_diag(N, tp.omega)
    R = np.zeros((tp.xyz.shape[0], nm), dtype=np.complex128)
    for s in range(0, tp.tets.shape[0], chunk):
        el = np.arange(s, min(s + chunk, tp.tets.shape[0]))
        tets = tp.tets[el]
        dN, vol, G = tp.dN[el], tp.vol[el], tp.G[el]
        pe = Phi[tets]                                     # [C,4,nm]
        ae = Av[tets]                                      # [C,4,3,nm]
        grad = np.einsum("caj,cam->cjm", dN, pe)           # dphi/dx_j
        r = np.zeros((el.size, 4, nm), dtype=np.complex128)
        w = vol / 4.0
        for q in range(4):
            lam = QP_BARY[q]
            aq = np.einsum("a,caim->cim", lam, ae)         # velocity modes at the point
            A = conv_matrix(aq)                            # [C,3,nm,nm]
            tau = tau_matrix(A, G, tp.kappa, tp.C_I)       # eq. (3D-tau)
            pq = np.einsum("a,cam->cm", lam, pe)
            res = om * pq + np.einsum("cjmn,cjn->cm", A, grad)
            T = np.einsum("cmn,cn->cm", tau, res)
            AT = np.einsum("cjmn,cn->cjm", A, T)
            r += w[:, None, None] * (lam[None, :, None] * res[:, None]
                                     - lam[None, :, None] * (om * T)[:, None]
                                     + np.einsum("caj,cjm->cam", dN, AT))
        r += (tp.kappa * vol)[:, None, None] * np.einsum("caj,cjm->cam", dN, grad)
        np.add.at(R, tets, r)
    R[tp.dmask] = 0.0
    if return_complex:
        return R
    return to_storage(R, N)
