"""Seeded problem set-ups: physical parameters, inflow waveforms, boundary data.

Input generation only.  The boundary data are the caller-side inputs of the
method: Fourier coefficients of the inlet waveform (the paper's g_n, computed
as (1/T) int g(t) e^{-i n w t} dt, section 2.4) and the Dirichlet values they
induce at inlet nodes.  Nothing here evaluates the GLS residual, its tangent
or tau.

Storage convention shared with both the CUDA path and the CPU checker: a
modal field is a float array ``y[V, 4, N, 2]`` -- node, field (u1, u2, u3,
p), mode n = 0..N-1, (real, imaginary).  The imaginary part of mode 0 is
carried but is always zero (the paper keeps it "to simplify
implementation", section 2.5.1).

Parameters follow the paper's diameter-based groups (section 3.1):
Re = rho U D / mu, Wo = D sqrt(rho omega / mu), with rho = 1, U = 1 (mean
inlet-1 velocity of mode 0) and D the inlet-1 diameter.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import meshgen as mg


@dataclass
class Case:
    mesh: mg.Mesh
    N: int
    rho: float
    mu: float
    omega: float
    C_I: float = 3.0
    c1: float = 1.5
    dirichlet_tags: tuple = (mg.TAG_WALL, mg.TAG_INLET1, mg.TAG_INLET2)
    resistance: dict = field(default_factory=dict)   # tag -> R
    backflow: dict = field(default_factory=dict)     # tag -> beta (backflow stabilisation)
    y0: np.ndarray | None = None                      # [V,4,N,2] float64 initial state
    dirichlet_mask: np.ndarray | None = None          # [V] bool
    info: dict = field(default_factory=dict)

    @property
    def nu(self) -> float:
        return self.mu / self.rho


def params_from_re_wo(Re: float, Wo: float, D: float, U: float = 1.0, rho: float = 1.0):
    mu = rho * U * D / Re
    omega = Wo * Wo * mu / (rho * D * D)
    return rho, mu, omega


def dirichlet_nodes(mesh: mg.Mesh, tags) -> np.ndarray:
    mask = np.zeros(mesh.n_nodes, dtype=bool)
    for t in tags:
        mask[mesh.bfaces[mesh.btag == t].ravel()] = True
    return mask


def nodes_with_tag(mesh: mg.Mesh, tag: int) -> np.ndarray:
    m = np.zeros(mesh.n_nodes, dtype=bool)
    m[mesh.bfaces[mesh.btag == tag].ravel()] = True
    return m


# ------------------------------------------------------------------ waveforms

def waveform_random(N: int, seed: int, amp: float = 0.2, mean: float = 1.0) -> np.ndarray:
    """Complex coefficients U_n, n = 0..N-1, amplitudes decaying like 1/n^2."""
    rng = np.random.default_rng(seed)
    c = np.zeros(N, dtype=np.complex128)
    c[0] = mean
    k = np.arange(1, N)
    c[1:] = amp * (rng.standard_normal(N - 1) + 1j * rng.standard_normal(N - 1)) / k ** 2
    return c


def waveform_fixed(amplitudes) -> np.ndarray:
    return np.asarray(amplitudes, dtype=np.complex128)


def womersley_profile(r: np.ndarray, R: float, Un: complex, n: int, omega: float, nu: float):
    """Axial velocity of fully developed pulsatile pipe flow for mode n with mean velocity Un.

    Boundary data for the pipe inlet; uses scipy's complex Bessel functions.
    """
    from scipy.special import jv

    if n == 0:
        return 2.0 * Un * (1.0 - (r / R) ** 2)
    alpha = R * np.sqrt(n * omega / nu)
    lam = (1j) ** 1.5 * alpha
    j0 = jv(0, lam)
    shape = 1.0 - jv(0, lam * r / R) / j0
    mean_shape = 1.0 - 2.0 * jv(1, lam) / (lam * j0)
    return Un * shape / mean_shape


def _set_mode(y, nodes, comp, n, val):
    y[nodes, comp, n, 0] = np.real(val)
    y[nodes, comp, n, 1] = 0.0 if n == 0 else np.imag(val)


# ------------------------------------------------------------------ cases

def pipe_case(N: int = 3, Re: float = 100.0, Wo: float = 5.0, amps=(1.0, 0.5, 0.25),
              mesh: mg.Mesh | None = None, profile: str = "womersley", **mesh_kw) -> Case:
    """Womersley pulsatile flow in a straight cylinder, zero-traction outlet."""
    mesh = mesh if mesh is not None else mg.pipe(**mesh_kw)
    R = mesh.info["R"]
    rho, mu, omega = params_from_re_wo(Re, Wo, D=2 * R)
    U = np.zeros(N, dtype=np.complex128)
    a = np.asarray(amps, dtype=np.complex128)
    U[: min(N, a.size)] = a[: min(N, a.size)]
    case = Case(mesh=mesh, N=N, rho=rho, mu=mu, omega=omega,
                dirichlet_tags=(mg.TAG_WALL, mg.TAG_INLET1))
    dmask = dirichlet_nodes(mesh, case.dirichlet_tags)
    wall = nodes_with_tag(mesh, mg.TAG_WALL)
    inlet = nodes_with_tag(mesh, mg.TAG_INLET1) & ~wall
    y0 = np.zeros((mesh.n_nodes, 4, N, 2))
    r = np.hypot(mesh.xyz[inlet, 0], mesh.xyz[inlet, 1])
    for n in range(N):
        if U[n] == 0:
            continue
        if profile == "womersley":
            w = womersley_profile(r, R, U[n], n, omega, mu / rho)
        else:
            w = 2.0 * U[n] * (1.0 - (r / R) ** 2)
        _set_mode(y0, inlet, 2, n, w)
    case.y0 = y0
    case.dirichlet_mask = dmask
    case.info = dict(kind="pipe", Re=Re, Wo=Wo, U=U, R=R, L=mesh.info["L"], profile=profile)
    return case


def junction_case(N: int = 7, Re: float = 500.0, Wo: float = 10.0, wave_seed: int = 100,
                  resistance: float = 1.0, mesh: mg.Mesh | None = None, amp: float = 0.2,
                  **mesh_kw) -> Case:
    """Fontan-like cross junction: parabolic inflow x random 1/k^2 waveform, resistance outlets."""
    mesh = mesh if mesh is not None else mg.junction(**mesh_kw)
    arms = {tag: (ax, sg, R) for ax, sg, R, tag in mg.JUNCTION_ARMS}
    D = 2 * arms[mg.TAG_INLET1][2]
    rho, mu, omega = params_from_re_wo(Re, Wo, D=D)
    res = {mg.TAG_OUTLET1: resistance, mg.TAG_OUTLET2: resistance} if resistance else {}
    case = Case(mesh=mesh, N=N, rho=rho, mu=mu, omega=omega,
                dirichlet_tags=(mg.TAG_WALL, mg.TAG_INLET1, mg.TAG_INLET2), resistance=res)
    dmask = dirichlet_nodes(mesh, case.dirichlet_tags)
    wall = nodes_with_tag(mesh, mg.TAG_WALL)
    y0 = np.zeros((mesh.n_nodes, 4, N, 2))
    waves = {}
    for k, tag in enumerate((mg.TAG_INLET1, mg.TAG_INLET2)):
        ax, sg, R = arms[tag]
        ai = mg._AX[ax]
        o = [d for d in range(3) if d != ai]
        nodes = nodes_with_tag(mesh, tag) & ~wall
        U = waveform_random(N, wave_seed + k, amp=amp)
        waves[tag] = U
        r = np.hypot(mesh.xyz[nodes, o[0]], mesh.xyz[nodes, o[1]])
        prof = np.clip(1.0 - (r / R) ** 2, 0.0, None)
        for n in range(N):
            # inflow points along -sg * axis (into the domain)
            _set_mode(y0, nodes, ai, n, -sg * 2.0 * U[n] * prof)
    case.y0 = y0
    case.dirichlet_mask = dmask
    case.info = dict(kind="junction", Re=Re, Wo=Wo, waves=waves, wave_seed=wave_seed, amp=amp)
    return case


# ------------------------------------------------------------------ learned-guess inputs

def surrogate_inputs(waves, Re: float, Wo: float, harmonics: int = 4) -> np.ndarray:
    """Network input for an inflow: Re and Im of harmonics 1..harmonics of every
    inlet waveform (complex coefficients indexed by mode), then (Re - 500) / 300
    and Wo / 10.  Two inlets with 4 harmonics give the 16 + 2 inputs of the
    junction surrogate."""
    x = []
    for U in waves:
        U = np.asarray(U, dtype=np.complex128)
        for n in range(1, harmonics + 1):
            c = U[n] if n < U.size else 0.0
            x += [np.real(c), np.imag(c)]
    x += [(Re - 500.0) / 300.0, Wo / 10.0]
    return np.asarray(x, dtype=np.float64)


# ------------------------------------------------------------------ random fields

def random_state(mesh: mg.Mesh, N: int, seed: int, scale_u: float = 1.0, scale_p: float = 1.0,
                 smooth: bool = True) -> np.ndarray:
    """Seeded modal field [V,4,N,2] with amplitudes decaying in n; Im of mode 0 is zero.

    ``smooth`` builds each mode from low-order polynomials of the coordinates
    plus small noise, so velocity gradients resemble a flow field.
    """
    rng = np.random.default_rng(seed)
    V = mesh.n_nodes
    y = np.zeros((V, 4, N, 2))
    x = mesh.xyz
    xc = (x - x.mean(axis=0)) / max(np.ptp(x, axis=0).max(), 1e-12)
    basis = np.column_stack([np.ones(V), xc, xc ** 2, xc[:, [0]] * xc[:, [1]], np.sin(3 * xc)])
    for f in range(4):
        s = scale_p if f == 3 else scale_u
        for n in range(N):
            for c in range(2):
                if n == 0 and c == 1:
                    continue
                if smooth:
                    coef = rng.standard_normal(basis.shape[1])
                    val = basis @ coef + 0.1 * rng.standard_normal(V)
                else:
                    val = rng.standard_normal(V)
                y[:, f, n, c] = s * val / (1.0 + n) ** 2
    return y
