"""Discrete residual (eq. Rmc) and tangent products (eq. K_mat), section 2.4.

For every element and quadrature point, in the paper's complex form
(modes -N+1..N-1):

  u^h, p^h at the point, grad u_i, grad p (constant on a P1 element)
  c_i  = A_j du_i/dx_j                          convective product, A_j = A(u_j)
  L_i  = rho Omega u_i + rho c_i + dp/dx_i       strong momentum residual; the
                                                 viscous second derivative is
                                                 dropped for linear shape
                                                 functions (section 2.4)
  T_i  = tau L_i                                 tau from eq. (3D-tau)

  r^m_{Ai} += w [rho N_A Omega u_i + rho N_A c_i - dN_A/dx_i p]
            + w mu dN_A/dx_j du_i/dx_j
            + w [(-Omega N_A) T_i + dN_A/dx_j (A_j T_i)]
  r^c_A    += w N_A du_i/dx_i + w (1/rho) dN_A/dx_i T_i

for A not on the Dirichlet boundary (momentum) and every A (continuity),
eq. (Rmc).  Neumann data: -int_{Gamma_h} N_A h n_i with h = 0 (traction
free) or, for a resistance outlet (an input of this build, not of the
paper), h_n = -R Q_n, Q_n = int_outlet u_n . n, which is linear in u.

Given A and tau, every term is linear in (u, p), so the residual equals the
"frozen" linear operator evaluated at its own linearisation point.  The
Jacobian-vector products follow eq. (K_mat), with A and tau frozen at the
linearisation state (section 2.4, remark 5):

  'frozen' : all blocks of eq. (K_mat) (K, G_i, D_j, L with their
             least-squares parts)
  'paper'  : least-squares parts dropped from G_i and D_j (section 2.5.2),
             i.e. the momentum least-squares term sees only the velocity part
             of L_i and the continuity least-squares term only dp/dx_i.
  'lin_a'  : 'frozen' plus the derivative of the convolution matrices
             (A_j is linear in u_j; only tau stays frozen).  Not a variant the
             paper uses; it is the exact derivative of the residual with tau
             held fixed, added for faster Newton convergence:
               + rho N_A A(v_j) du0_i/dx_j                  (Galerkin)
               + tau-weighted rho A(v_j) du0_i/dx_j in L_i   (least squares)
               + dN_A/dx_j A(v_j) T0_i                       (test-function change)
             with T0_i = tau L_i(u0, p0).

Pseudo-time stepping (section 2.5.3) adds (N_A, c1 rho / dt N_B I) to K,
i.e. ``mass_coef * M v`` on the momentum rows with the consistent mass M.

Rows and unknowns fixed by the method: momentum rows of Dirichlet nodes
(residual zero), Dirichlet velocity unknowns (tangent input ignored), the
imaginary part of mode 0 (always zero).

Elements are accumulated in mesh order (no colouring).

Pinned by: tests/test_oracle_operator.py -- steady limit equals the
independent SUPG/PSPG residual of eq. (NSt-weak); conjugate symmetry of the
residual (section 3.3); central differences of the residual equal the
'frozen' product at u = 0 and in the pressure unknowns at any state (A and
tau do not depend on p); the dense tangent built from eq. (K_mat) equals the
products column by column (tests/test_oracle_assemble.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .geometry import QP_BARY, face_normals_areas, tet_geometry
from .spectral import conv_matrix, omega_diag, to_complex, to_storage
from .tau import tau_matrix


@dataclass
class Problem:
    xyz: np.ndarray
    tets: np.ndarray
    N: int
    rho: float
    mu: float
    omega: float
    C_I: float
    dmask: np.ndarray                     # [V] bool, Dirichlet velocity nodes
    outlets: list = field(default_factory=list)   # [(faces [F,3], R)]
    backflow: list = field(default_factory=list)  # [(faces [F,3], beta)]
    dN: np.ndarray = None
    vol: np.ndarray = None
    G: np.ndarray = None

    @property
    def nm(self) -> int:
        return 2 * self.N - 1

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]


def make_problem(xyz, tets, N, rho, mu, omega, dmask, C_I=3.0, outlets=(), backflow=()) -> Problem:
    dN, vol, G = tet_geometry(np.asarray(xyz, np.float64), np.asarray(tets))
    return Problem(xyz=np.asarray(xyz, np.float64), tets=np.asarray(tets, np.int64), N=N,
                   rho=rho, mu=mu, omega=omega, C_I=C_I, dmask=np.asarray(dmask, bool),
                   outlets=list(outlets), backflow=list(backflow), dN=dN, vol=vol, G=G)


def problem_from_case(case) -> Problem:
    m = case.mesh
    outlets = [(m.bfaces[m.btag == tag], R) for tag, R in case.resistance.items()]
    backflow = [(m.bfaces[m.btag == tag], b) for tag, b in getattr(case, "backflow", {}).items()]
    return make_problem(m.xyz, m.tets, case.N, case.rho, case.mu, case.omega,
                        case.dirichlet_mask, case.C_I, outlets, backflow)


def free_mask(prob: Problem) -> np.ndarray:
    """Storage-shaped [V,4,N,2] mask of unknowns that the method solves for."""
    f = np.ones((prob.n_nodes, 4, prob.N, 2), dtype=bool)
    f[prob.dmask, 0:3] = False
    f[:, :, 0, 1] = False
    return f


@dataclass
class Linearization:
    elems: np.ndarray          # element ids covered
    A: np.ndarray              # [E',4,3,nm,nm] convolution matrices of u0 at each point
    tau: np.ndarray            # [E',4,nm,nm]
    grad_u0: np.ndarray = None  # [E',3(i),3(j),nm] du0_i/dx_j ('lin_a' only)
    T0: np.ndarray = None       # [E',4,3,nm] tau L_i(u0, p0) ('lin_a' only)
    Bneg: list = None           # per backflow face set: [F,3,nm,nm] |A_n|_- at each face point


def linearize(prob: Problem, y0: np.ndarray, elems=None, tau_state=None) -> Linearization:
    """Freeze A_j and tau at the state y0 (storage layout).

    ``tau_state`` (optional) evaluates tau at another state, used to build a
    residual with tau held fixed while A follows y0.
    """
    elems = np.arange(prob.tets.shape[0]) if elems is None else np.asarray(elems)
    Y = to_complex(y0, prob.N)                             # [V,4,nm]
    ue = Y[prob.tets[elems], 0:3]                          # [E',4,3,nm]
    pe = Y[prob.tets[elems], 3]
    uq = np.einsum("qa,eaim->eqim", QP_BARY, ue)           # u0 at each point
    A = conv_matrix(uq)                                    # [E',4,3,nm,nm]
    G = np.broadcast_to(prob.G[elems][:, None], (elems.size, 4, 3, 3))
    if tau_state is None:
        tau = tau_matrix(A, G, prob.mu / prob.rho, prob.C_I)
    else:
        tau = linearize(prob, tau_state, elems).tau
    dN = prob.dN[elems]
    grad_u0 = np.einsum("eaj,eaim->eijm", dN, ue)
    grad_p0 = np.einsum("eaj,eam->ejm", dN, pe)
    om = omega_diag(prob.N, prob.omega)
    conv = np.einsum("eqjmn,eijn->eqim", A, grad_u0)
    L0 = prob.rho * om * uq + prob.rho * conv + grad_p0[:, None]
    T0 = np.einsum("eqmn,eqin->eqim", tau, L0)
    Bneg = [_backflow_matrices(prob, Y[:, 0:3], faces) for faces, _ in prob.backflow]
    return Linearization(elems=elems, A=A, tau=tau, grad_u0=grad_u0, T0=T0, Bneg=Bneg)


# 3-point rule of degree 2 on a triangle: barycentric coordinates, weights area/3
FACE_BARY = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])


def _backflow_matrices(prob: Problem, U: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """|A_n|_- = (A_n - |A_n|)/2 at every face point, A_n = A_i n_i = A(u . n) (section 2.6).

    |A_n| is taken through the eigenpairs of the Hermitian A_n, as the paper
    describes (remark 1 of section 2.6).  Returns [F, 3, nm, nm].
    """
    n, _ = face_normals_areas(prob.xyz, faces)
    un = np.einsum("fi,fbim->fbm", n, U[faces])            # u . n at the face vertices
    ung = np.einsum("gb,fbm->fgm", FACE_BARY, un)          # at the 3 face points
    An = conv_matrix(ung)                                   # [F,3,nm,nm]
    An = 0.5 * (An + np.conj(np.swapaxes(An, -1, -2)))
    lam, V = np.linalg.eigh(An)
    neg = np.minimum(lam, 0.0)
    return np.einsum("...mk,...k,...nk->...mn", V, neg, np.conj(V))


def _outlet_flux(prob: Problem, U: np.ndarray, faces: np.ndarray):
    """Q_n = int_outlet u_n . n dGamma for every mode, plus the nodal weights."""
    n, area = face_normals_areas(prob.xyz, faces)
    w = (area / 3.0)[:, None] * n                          # [F,3] = int N_a n_i per face vertex
    Q = np.einsum("fi,fbim->m", w, U[faces])               # sum over the 3 face vertices
    return Q, w


def apply(prob: Problem, lin: Linearization, y: np.ndarray, variant: str = "frozen",
          mask_dirichlet_input: bool = False, mass_coef: float = 0.0,
          return_complex: bool = False, chunk: int = 2048):
    """Apply the operator with A and tau frozen in ``lin`` to the state ``y``.

    variant 'frozen' with y equal to the linearisation state is the residual
    of eq. (Rmc); with a perturbation it is the eq. (K_mat) tangent product.
    """
    N, rho, mu = prob.N, prob.rho, prob.mu
    nm = prob.nm
    Y = to_complex(y, N)                                    # [V,4,nm]
    if mask_dirichlet_input:
        Y = Y.copy()
        Y[prob.dmask, 0:3] = 0.0
    om = omega_diag(N, prob.omega)                          # [nm]
    Ru = np.zeros((prob.n_nodes, 3, nm), dtype=np.complex128)
    Rc = np.zeros((prob.n_nodes, nm), dtype=np.complex128)
    elems = lin.elems
    for s in range(0, elems.size, chunk):
        sl = slice(s, min(s + chunk, elems.size))
        el = elems[sl]
        tets = prob.tets[el]
        dN = prob.dN[el]                                    # [C,4,3]
        vol = prob.vol[el]
        ue = Y[tets, 0:3]                                   # [C,4(a),3(i),nm]
        pe = Y[tets, 3]                                     # [C,4,nm]
        grad_u = np.einsum("caj,caim->cijm", dN, ue)        # du_i/dx_j
        grad_p = np.einsum("caj,cam->cjm", dN, pe)          # dp/dx_j
        div = np.einsum("ciim->cm", grad_u)
        rm = np.zeros((el.size, 4, 3, nm), dtype=np.complex128)
        rc = np.zeros((el.size, 4, nm), dtype=np.complex128)
        for q in range(4):
            lam = QP_BARY[q]                                # N_a at the point
            w = vol / 4.0
            uq = np.einsum("a,caim->cim", lam, ue)
            pq = np.einsum("a,cam->cm", lam, pe)
            A = lin.A[sl, q]                                # [C,3(j),nm,nm]
            tau = lin.tau[sl, q]                            # [C,nm,nm]
            conv = np.einsum("cjmn,cijn->cim", A, grad_u)   # c_i = A_j du_i/dx_j
            if variant == "lin_a":
                Av = conv_matrix(uq)                        # A(v_j) at the point
                conv = conv + np.einsum("cjmn,cijn->cim", Av, lin.grad_u0[sl])
            Lu = rho * om * uq + rho * conv                 # velocity part of L_i
            Lp = grad_p                                     # pressure part of L_i
            # Galerkin terms of eq. (Rmc)
            rm += w[:, None, None, None] * (
                rho * lam[None, :, None, None] * (om * uq + conv)[:, None]
                - dN[:, :, :, None] * pq[:, None, None, :])
            rc += w[:, None, None] * lam[None, :, None] * div[:, None, :]
            # least-squares terms of eq. (Rmc)
            if variant in ("frozen", "lin_a"):
                Tm = np.einsum("cmn,cin->cim", tau, Lu + Lp)
                Tc = Tm
            elif variant == "paper":
                Tm = np.einsum("cmn,cin->cim", tau, Lu)
                Tc = np.einsum("cmn,cin->cim", tau, Lp)
            else:
                raise ValueError(variant)
            AT = np.einsum("cjmn,cin->cjim", A, Tm)        # A_j T_i
            if variant == "lin_a":
                AT = AT + np.einsum("cjmn,cin->cjim", Av, lin.T0[sl, q])
            rm += w[:, None, None, None] * (
                -lam[None, :, None, None] * (om * Tm)[:, None]
                + np.einsum("caj,cjim->caim", dN, AT))
            rc += (w / rho)[:, None, None] * np.einsum("cai,cim->cam", dN, Tc)
        # viscous Galerkin term (constant integrand on a P1 element)
        rm += (mu * vol)[:, None, None, None] * np.einsum("caj,cijm->caim", dN, grad_u)
        if mass_coef:
            Mab = (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))
            rm += mass_coef * np.einsum("cab,cbim->caim", Mab, ue)
        np.add.at(Ru, tets, rm)
        np.add.at(Rc, tets, rc)
    # Neumann term, resistance outlets: -int N_A h n_i with h = -R Q
    for faces, R in prob.outlets:
        Q, w = _outlet_flux(prob, Y[:, 0:3], faces)
        contrib = R * w[:, None, :, None] * Q[None, None, None, :]    # [F,1,3,nm]
        np.add.at(Ru, faces, np.broadcast_to(contrib, (faces.shape[0], 3, 3, nm)))
    # backflow stabilisation (section 2.6): the term (w, (rho/2) beta |A_n|_- u)_Gh
    # on the right-hand side of eq. (NS-weak), i.e. -int N_A (rho/2) beta |A_n|_- u_i
    for (faces, beta), B in zip(prob.backflow, lin.Bneg or []):
        _, area = face_normals_areas(prob.xyz, faces)
        ug = np.einsum("gb,fbim->fgim", FACE_BARY, Y[faces, 0:3])   # u at the face points
        z = np.einsum("fgmn,fgin->fgim", B, ug)
        contrib = -0.5 * rho * beta * (area / 3.0)[:, None, None, None, None] * \
            np.einsum("gb,fgim->fbim", FACE_BARY, z)[:, None]       # [F,1,3(b),3(i),nm]
        np.add.at(Ru, faces, contrib[:, 0])
    Rout = np.concatenate([Ru, Rc[:, None, :]], axis=1)    # [V,4,nm]
    if return_complex:
        return Rout
    Rout[prob.dmask, 0:3] = 0.0
    return to_storage(Rout, N)


def residual(prob: Problem, y: np.ndarray, return_complex: bool = False, elems=None):
    """r(y) of eq. (Rmc): A and tau evaluated at y itself."""
    lin = linearize(prob, y, elems)
    return apply(prob, lin, y, "frozen", return_complex=return_complex)


def jvp(prob: Problem, lin: Linearization, v: np.ndarray, variant: str = "paper",
        mass_coef: float = 0.0) -> np.ndarray:
    """H v with A and tau frozen at ``lin`` (eq. K_mat; 'paper' drops LS from G and D)."""
    return apply(prob, lin, v, variant, mask_dirichlet_input=True, mass_coef=mass_coef)


def element_sample_for_nodes(prob: Problem, nodes: np.ndarray) -> np.ndarray:
    """Elements touching any of ``nodes``: enough to evaluate the operator there exactly."""
    hit = np.isin(prob.tets, nodes).any(axis=1)
    return np.nonzero(hit)[0]
