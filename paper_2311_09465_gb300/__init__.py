"""Python binding of ``libtsgls`` (GB300 time-spectral GLS Navier-Stokes).

Argument marshalling only: every step of the operator and of the solve runs
in the CUDA library (``include/tsgls.h``).  Modal fields are CUDA tensors of
shape [V, 4, N, 2] (node, field u1/u2/u3/p, mode, re/im), float32 or float64,
contiguous.  There is no CPU fallback: the first call loads the library
and raises ImportError if it is missing (build it with
``python -m paper_2311_09465_gb300.build``).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtsgls.so")

TS_OK, TS_ERR_ARG, TS_ERR_CUDA, TS_ERR_OOM, TS_ERR_NOCONV, TS_ERR_NAN, TS_ERR_UNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
TS_BC_DIRICHLET, TS_BC_TRACTION, TS_BC_RESISTANCE, TS_BC_BACKFLOW = 1, 2, 3, 4
TS_PROFILE_PARABOLIC, TS_PROFILE_WOMERSLEY = 1, 2
PROFILES = {"parabolic": TS_PROFILE_PARABOLIC, "womersley": TS_PROFILE_WOMERSLEY}
TS_JVP_PAPER, TS_JVP_FROZEN, TS_JVP_LIN_A, TS_JVP_EXACT = 0, 1, 2, 3
VARIANTS = {"paper": TS_JVP_PAPER, "frozen": TS_JVP_FROZEN, "lin_a": TS_JVP_LIN_A, "exact": TS_JVP_EXACT}
TS_OPT_TAU64, TS_OPT_FP32_TANGENT, TS_OPT_ELEMENT64, TS_OPT_TAU_WARM = 1, 2, 3, 4
TS_ELEMENT64_NATIVE, TS_ELEMENT64_DOUBLEFLOAT = 0, 1
ELEMENT64 = {"native": TS_ELEMENT64_NATIVE, "doublefloat": TS_ELEMENT64_DOUBLEFLOAT}
TS_TAU64_REFINE, TS_TAU64_DOUBLEFLOAT, TS_TAU64_JACOBI = 0, 1, 2
TAU64 = {"refine": TS_TAU64_REFINE, "doublefloat": TS_TAU64_DOUBLEFLOAT, "jacobi": TS_TAU64_JACOBI}
SUPPORTED_N = (1, 2, 3, 4, 5, 7, 10, 15)


class TsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tsgls error {code}: {msg}")
        self.code = code


class ts_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("rho", ctypes.c_double), ("mu", ctypes.c_double),
                ("omega", ctypes.c_double), ("C_I", ctypes.c_double), ("c1", ctypes.c_double),
                ("dt_pseudo", ctypes.c_double), ("jvp_variant", ctypes.c_int)]


class ts_solve_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("r_ref", ctypes.c_double),
                ("max_steps", ctypes.c_int), ("krylov", ctypes.c_int), ("eps_ls", ctypes.c_double),
                ("max_matvec", ctypes.c_int), ("verbose", ctypes.c_int), ("precond", ctypes.c_int),
                ("ser", ctypes.c_double), ("dt_max", ctypes.c_double), ("reject", ctypes.c_double)]


class ts_solve_report(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("matvecs", ctypes.c_int), ("r_ref", ctypes.c_double),
                ("r_final", ctypes.c_double), ("seconds", ctypes.c_double),
                ("t_residual", ctypes.c_double), ("t_jvp", ctypes.c_double),
                ("t_krylov", ctypes.c_double), ("hist_len", ctypes.c_int),
                ("hist", ctypes.c_double * 512), ("rejected", ctypes.c_int),
                ("t_precond", ctypes.c_double), ("t_tau", ctypes.c_double),
                ("n_residual", ctypes.c_int)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "hist"}
        d["hist"] = list(self.hist[: self.hist_len])
        return d


_lib = None


def lib() -> ctypes.CDLL:
    """Load libtsgls.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtsgls.so not built ({LIB_PATH}); run python -m paper_2311_09465_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32p, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
    L.ts_mesh_load.argtypes = [dp, i64, i32p, i64, i32p, i32p, i64, ctypes.POINTER(vp)]
    L.ts_mesh_free.argtypes = [vp]
    L.ts_mesh_free.restype = None
    L.ts_mesh_colors.argtypes = [vp]
    L.ts_mesh_node_colours.argtypes = [vp, i32p]
    L.ts_problem_create.argtypes = [vp, ctypes.POINTER(ts_params), ctypes.POINTER(vp)]
    L.ts_problem_free.argtypes = [vp]
    L.ts_problem_free.restype = None
    L.ts_problem_set.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.ts_set_bc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.ts_problem_option.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.ts_set_inlet.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, dp]
    L.ts_inlet_info.argtypes = [vp, ctypes.c_int, dp]
    L.ts_initial_guess.argtypes = [vp, vp, ctypes.c_int, vp]
    L.ts_residual.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    L.ts_jvp.argtypes = [vp, vp, vp, ctypes.c_int, vp]
    L.ts_block_diagonal.argtypes = [vp, vp, ctypes.c_int, vp]
    L.ts_precond_setup.argtypes = [vp, ctypes.c_int, vp]
    L.ts_precond_apply.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    L.ts_assemble.argtypes = [vp, vp]
    L.ts_spmv.argtypes = [vp, vp, vp, vp]
    L.ts_assembled_bytes.argtypes = [vp]
    L.ts_assembled_bytes.restype = ctypes.c_int64
    L.ts_mesh_connections.argtypes = [vp]
    L.ts_mesh_connections.restype = ctypes.c_int64
    L.ts_residual_noalloc.argtypes = [vp, vp, vp, vp]
    L.ts_solve.argtypes = [vp, vp, ctypes.POINTER(ts_solve_opts), ctypes.POINTER(ts_solve_report), vp]
    fp, u64 = ctypes.POINTER(ctypes.c_float), ctypes.c_uint64
    L.ts_surrogate_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, u64,
                                      ctypes.POINTER(vp)]
    L.ts_surrogate_free.argtypes = [vp]
    L.ts_surrogate_free.restype = None
    L.ts_surrogate_num_params.argtypes = [vp]
    L.ts_surrogate_num_params.restype = ctypes.c_int64
    L.ts_surrogate_get_params.argtypes = [vp, fp, i64]
    L.ts_surrogate_set_params.argtypes = [vp, fp, i64]
    L.ts_surrogate_forward.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    L.ts_surrogate_gradient.argtypes = [vp, vp, vp, ctypes.c_int, vp, dp, vp]
    L.ts_surrogate_adam.argtypes = [vp, vp, ctypes.c_double, vp]
    L.ts_surrogate_fit_basis.argtypes = [vp, vp, ctypes.c_int, vp]
    L.ts_surrogate_basis_rank.argtypes = [vp, dp]
    L.ts_surrogate_coefficients.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    L.ts_surrogate_train.argtypes = [vp, fp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     u64, dp, vp]
    L.ts_surrogate_guess.argtypes = [vp, vp, fp, vp, vp]
    L.ts_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    L.ts_batch_free.argtypes = [vp]
    L.ts_batch_free.restype = None
    L.ts_batch_jvp.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.ts_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ts_solve_opts),
                                 ctypes.POINTER(ts_solve_report), vp]
    L.ts_batch_launch_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.ts_tracer_create.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(vp)]
    L.ts_tracer_free.argtypes = [vp]
    L.ts_tracer_free.restype = None
    L.ts_tracer_set_dirichlet.argtypes = [vp, ctypes.c_int]
    L.ts_tracer_residual.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp]
    L.ts_tracer_set_stabilised.argtypes = [vp, ctypes.c_int]
    L.ts_tracer_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), dp, vp]
    L.ts_last_error.restype = ctypes.c_char_p
    L.ts_version.restype = ctypes.c_char_p
    L.ts_launch_count.restype = ctypes.c_int64
    L.ts_stage_times.argtypes = [vp, dp]
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise TsError(rc, lib().ts_last_error().decode())
    return rc


def ts_last_error() -> str:
    return lib().ts_last_error().decode()


def ts_version() -> str:
    return lib().ts_version().decode()


def ts_launch_count() -> int:
    return int(lib().ts_launch_count())


def ts_stage_times(prob) -> dict:
    """Device milliseconds of the last residual's tau kernel and element pass and
    of the last FP32 tangent product's element kernel (-1: not run yet)."""
    out = (ctypes.c_double * 3)()
    _check(lib().ts_stage_times(prob, out))
    return {"tau_ms": out[0], "residual_element_ms": out[1], "jvp_element_ms": out[2]}


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _field_ptr(t, precision=None):
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("modal fields must be contiguous CUDA tensors")
    p = 64 if t.dtype == torch.float64 else 32 if t.dtype == torch.float32 else None
    if p is None:
        raise ValueError("modal fields must be float32 or float64")
    if precision is not None and precision != p:
        raise ValueError("tensor dtype does not match precision")
    return ctypes.c_void_p(t.data_ptr()), p


# ------------------------------------------------------------------ C ABI mirrors

def ts_mesh_load(xyz, tets, bfaces, btag):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    bfaces = np.ascontiguousarray(bfaces, dtype=np.int32)
    btag = np.ascontiguousarray(btag, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib().ts_mesh_load(xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), xyz.shape[0],
                              tets.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tets.shape[0],
                              bfaces.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              btag.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), bfaces.shape[0],
                              ctypes.byref(out)))
    return out


def ts_mesh_free(mesh):
    lib().ts_mesh_free(mesh)


def ts_mesh_colors(mesh) -> int:
    n = lib().ts_mesh_colors(mesh)
    if n < 0:
        _check(n)
    return n


def ts_mesh_node_colours(mesh, n_nodes=None):
    """Number of node colours; with n_nodes, also each node's colour (int32 array)."""
    if n_nodes is None:
        n = lib().ts_mesh_node_colours(mesh, None)
        if n < 0:
            _check(n)
        return n
    out = np.zeros(int(n_nodes), dtype=np.int32)
    n = lib().ts_mesh_node_colours(mesh, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if n < 0:
        _check(n)
    return n, out


def ts_problem_create(mesh, params: ts_params):
    out = ctypes.c_void_p()
    _check(lib().ts_problem_create(mesh, ctypes.byref(params), ctypes.byref(out)))
    return out


def ts_problem_free(prob):
    lib().ts_problem_free(prob)


def ts_problem_set(prob, dt_pseudo: float, jvp_variant: int):
    _check(lib().ts_problem_set(prob, dt_pseudo, jvp_variant))


def ts_problem_option(prob, key: int, value: int):
    _check(lib().ts_problem_option(prob, key, value))


def ts_set_bc(prob, tag: int, kind: int, value: float = 0.0):
    _check(lib().ts_set_bc(prob, tag, kind, value))


def ts_set_inlet(prob, tag: int, Qn, profile="parabolic", centre=None, direction=None, radius=None):
    """Inlet Dirichlet data from complex flow-rate coefficients Qn (modes 0..N-1);
    the inlet geometry is derived from the mesh unless centre, direction (into the
    domain) and radius are all given."""
    q = np.asarray(Qn, dtype=np.complex128)
    buf = np.ascontiguousarray(np.stack([q.real, q.imag], axis=1), dtype=np.float64)
    geo = None
    if centre is not None:
        gbuf = np.ascontiguousarray(np.concatenate([np.asarray(centre, np.float64),
                                                    np.asarray(direction, np.float64), [float(radius)]]))
        geo = gbuf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(lib().ts_set_inlet(prob, tag, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              PROFILES[profile] if isinstance(profile, str) else int(profile), geo))


def ts_inlet_info(prob, tag: int) -> dict:
    out = np.zeros(7)
    _check(lib().ts_inlet_info(prob, tag, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return {"centre": out[0:3].copy(), "direction": out[3:6].copy(), "radius": float(out[6])}


def ts_initial_guess(prob, y, stream=None):
    py, p = _field_ptr(y)
    _check(lib().ts_initial_guess(prob, py, p, _stream_ptr(stream)))
    return y


def ts_residual(prob, y, r, precision=None, stream=None):
    py, p = _field_ptr(y, precision)
    pr, _ = _field_ptr(r, p)
    _check(lib().ts_residual(prob, py, pr, p, _stream_ptr(stream)))
    return r


def ts_residual_noalloc(prob, y, r, stream=None):
    """FP32 residual that allocates no device memory (fixed 32 MiB scratch)."""
    py, _ = _field_ptr(y, 32)
    pr, _ = _field_ptr(r, 32)
    _check(lib().ts_residual_noalloc(prob, py, pr, _stream_ptr(stream)))
    return r


def ts_jvp(prob, v, hv, precision=None, stream=None):
    pv, p = _field_ptr(v, precision)
    ph, _ = _field_ptr(hv, p)
    _check(lib().ts_jvp(prob, pv, ph, p, _stream_ptr(stream)))
    return hv


def ts_block_diagonal(prob, out, invert=False, stream=None):
    """Nodal diagonal blocks of the tangent into out (CUDA float32 [V, 8N, 8N]);
    invert: their inverses, column-major (see include/tsgls.h)."""
    import torch
    if not out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA float32 tensor")
    _check(lib().ts_block_diagonal(prob, ctypes.c_void_p(out.data_ptr()), int(bool(invert)),
                                   _stream_ptr(stream)))
    return out


def ts_precond_setup(prob, kind, stream=None):
    """Builds the block preconditioner kind 2 (block Jacobi) or 3 (symmetric
    block Gauss-Seidel) at the state of the last residual."""
    _check(lib().ts_precond_setup(prob, int(kind), _stream_ptr(stream)))


def ts_precond_apply(prob, kind, x, z, stream=None):
    """z = P^{-1} x with the preconditioner last built for kind (CUDA float64 fields)."""
    import torch
    for t in (x, z):
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError("x and z must be contiguous CUDA float64 tensors")
    _check(lib().ts_precond_apply(prob, int(kind), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                  _stream_ptr(stream)))
    return z


def ts_assemble(prob, stream=None):
    _check(lib().ts_assemble(prob, _stream_ptr(stream)))


def ts_spmv(prob, v, hv, stream=None):
    pv, _ = _field_ptr(v, 32)
    ph, _ = _field_ptr(hv, 32)
    _check(lib().ts_spmv(prob, pv, ph, _stream_ptr(stream)))
    return hv


def ts_assembled_bytes(prob) -> int:
    n = int(lib().ts_assembled_bytes(prob))
    if n < 0:
        _check(n)
    return n


def ts_mesh_connections(mesh) -> int:
    n = int(lib().ts_mesh_connections(mesh))
    if n < 0:
        _check(n)
    return n


def ts_solve(prob, y, opts: ts_solve_opts, stream=None, raise_on_noconv=True) -> dict:
    py, p = _field_ptr(y, 64)
    rep = ts_solve_report()
    rc = lib().ts_solve(prob, py, ctypes.byref(opts), ctypes.byref(rep), _stream_ptr(stream))
    d = rep.to_dict()
    d["status"] = rc
    if rc != 0 and (raise_on_noconv or rc != TS_ERR_NOCONV):
        raise TsError(rc, lib().ts_last_error().decode())
    return d


# ------------------------------------------------------------------ convenience

class GLSProblem:
    """Mesh + problem handles for a seeded case (``workloads.cases.Case``)."""

    def __init__(self, case, variant="lin_a", dt_pseudo=math.inf, tau64="doublefloat",
                 fp32_tangent="single", element64=None):
        m = case.mesh
        self.case = case
        self.N = case.N
        self.n_nodes = m.n_nodes
        self.mesh = ts_mesh_load(m.xyz, m.tets, m.bfaces, m.btag)
        prm = ts_params(N=case.N, rho=case.rho, mu=case.mu, omega=case.omega, C_I=case.C_I,
                        c1=case.c1, dt_pseudo=dt_pseudo, jvp_variant=VARIANTS[variant])
        self.prob = ts_problem_create(self.mesh, prm)
        for tag in case.dirichlet_tags:
            ts_set_bc(self.prob, tag, TS_BC_DIRICHLET)
        for tag, R in case.resistance.items():
            ts_set_bc(self.prob, tag, TS_BC_RESISTANCE, R)
        for tag, beta in getattr(case, "backflow", {}).items():
            ts_set_bc(self.prob, tag, TS_BC_BACKFLOW, beta)
        self.option(tau64=tau64, fp32_tangent=fp32_tangent, element64=element64)

    def option(self, tau64=None, fp32_tangent=None, element64=None, tau_warm=None):
        """tau64: "refine" | "doublefloat" | "jacobi"; fp32_tangent: "single" | "coloured";
        element64: "native" | "doublefloat"; tau_warm: bool (warm-started tau eigensolve)."""
        if tau_warm is not None:
            ts_problem_option(self.prob, TS_OPT_TAU_WARM, int(bool(tau_warm)))
        if element64 is not None:
            ts_problem_option(self.prob, TS_OPT_ELEMENT64, ELEMENT64[element64])
        if tau64 is not None:
            ts_problem_option(self.prob, TS_OPT_TAU64, TAU64[tau64])
        if fp32_tangent is not None:
            ts_problem_option(self.prob, TS_OPT_FP32_TANGENT,
                              {"single": 0, "coloured": 1}[fp32_tangent])

    def set_inlet(self, tag, Qn, profile="parabolic", centre=None, direction=None, radius=None):
        ts_set_inlet(self.prob, tag, Qn, profile, centre, direction, radius)

    def inlet_info(self, tag):
        return ts_inlet_info(self.prob, tag)

    def initial_guess(self, dtype=None, stream=None):
        """The paper's initial guess with the inlet data of set_inlet (new CUDA tensor)."""
        import torch
        y = self.field(torch.float64 if dtype is None else dtype)
        return ts_initial_guess(self.prob, y, stream)

    def set(self, dt_pseudo=math.inf, variant="lin_a"):
        ts_problem_set(self.prob, dt_pseudo, VARIANTS[variant])

    def colors(self):
        return ts_mesh_colors(self.mesh)

    def node_colours(self):
        """(number of node colours, each node's colour)."""
        return ts_mesh_node_colours(self.mesh, self.n_nodes)

    def precond_setup(self, kind, stream=None):
        ts_precond_setup(self.prob, kind, stream)

    def precond_apply(self, kind, x, z=None, stream=None):
        z = self.field(x.dtype, x.device) if z is None else z
        return ts_precond_apply(self.prob, kind, x, z, stream)

    def field(self, dtype, device="cuda"):
        import torch
        return torch.zeros((self.n_nodes, 4, self.N, 2), dtype=dtype, device=device)

    def residual(self, y, r=None, stream=None):
        r = self.field(y.dtype, y.device) if r is None else r
        return ts_residual(self.prob, y, r, stream=stream)

    def jvp(self, v, hv=None, stream=None):
        hv = self.field(v.dtype, v.device) if hv is None else hv
        return ts_jvp(self.prob, v, hv, stream=stream)

    def assemble(self, stream=None):
        ts_assemble(self.prob, stream)

    def spmv(self, v, hv=None, stream=None):
        hv = self.field(v.dtype, v.device) if hv is None else hv
        return ts_spmv(self.prob, v, hv, stream)

    def assembled_bytes(self):
        return ts_assembled_bytes(self.prob)

    def block_diagonal(self, invert=False, stream=None):
        import torch
        nb = 8 * self.N
        out = torch.empty((self.n_nodes, nb, nb), dtype=torch.float32, device="cuda")
        return ts_block_diagonal(self.prob, out, invert, stream)

    def solve(self, y, precision=64, tol=1e-8, r_ref=0.0, max_steps=200, krylov=100,
              eps_ls=0.05, max_matvec=10000, verbose=False, stream=None, raise_on_noconv=True,
              precond=1, ser=0.0, dt_max=0.0, reject=4.0):
        opts = ts_solve_opts(precision=precision, tol=tol, r_ref=r_ref, max_steps=max_steps,
                             krylov=krylov, eps_ls=eps_ls, max_matvec=max_matvec,
                             verbose=int(verbose), precond=int(precond), ser=float(ser),
                             dt_max=float(dt_max), reject=float(reject))
        return ts_solve(self.prob, y, opts, stream=stream, raise_on_noconv=raise_on_noconv)

    def close(self):
        if getattr(self, "prob", None):
            ts_problem_free(self.prob)
            self.prob = None
        if getattr(self, "mesh", None):
            ts_mesh_free(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batched solve

def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])


def ts_batch_create(probs):
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(probs))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in probs])
    _check(lib().ts_batch_create(arr, len(probs), ctypes.byref(h)))
    return h


def ts_batch_free(batch):
    lib().ts_batch_free(batch)


def ts_batch_jvp(batch, vs, hvs, stream=None):
    _check(lib().ts_batch_jvp(batch, _ptr_array([v.data_ptr() for v in vs]),
                              _ptr_array([h.data_ptr() for h in hvs]), _stream_ptr(stream)))
    return hvs


def ts_batch_solve(batch, ys, opts: ts_solve_opts, stream=None, raise_on_noconv=True):
    reps = (ts_solve_report * len(ys))()
    rc = lib().ts_batch_solve(batch, _ptr_array([y.data_ptr() for y in ys]), ctypes.byref(opts), reps,
                              _stream_ptr(stream))
    out = [r.to_dict() for r in reps]
    for d in out:
        d["status"] = rc
    if rc != 0 and (raise_on_noconv or rc != TS_ERR_NOCONV):
        raise TsError(rc, lib().ts_last_error().decode())
    return out


def ts_batch_launch_shape(batch):
    w, b = ctypes.c_int(), ctypes.c_int()
    tuned = lib().ts_batch_launch_shape(batch, ctypes.byref(w), ctypes.byref(b))
    return {"warps_per_block": w.value, "blocks": b.value, "tuned": bool(tuned)}


class Batch:
    """Lockstep mixed-precision solve of several ``GLSProblem`` instances."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.h = ts_batch_create([p.prob for p in self.problems])

    def jvp(self, vs, hvs=None, stream=None):
        hvs = [p.field(v.dtype, v.device) for p, v in zip(self.problems, vs)] if hvs is None else hvs
        return ts_batch_jvp(self.h, vs, hvs, stream)

    def solve(self, ys, tol=1e-8, r_ref=0.0, max_steps=200, krylov=100, eps_ls=0.05, max_matvec=10000,
              precond=1, ser=0.0, dt_max=0.0, stream=None, raise_on_noconv=True):
        opts = ts_solve_opts(precision=32, tol=tol, r_ref=r_ref, max_steps=max_steps, krylov=krylov,
                             eps_ls=eps_ls, max_matvec=max_matvec, verbose=0, precond=int(precond),
                             ser=float(ser), dt_max=float(dt_max))
        return ts_batch_solve(self.h, ys, opts, stream, raise_on_noconv)

    def launch_shape(self):
        return ts_batch_launch_shape(self.h)

    def close(self):
        if getattr(self, "h", None):
            ts_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ learned initial guess

def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def ts_surrogate_create(n_in, hidden, n_hidden_layers, n_out, n_dof, seed=0):
    h = ctypes.c_void_p()
    _check(lib().ts_surrogate_create(n_in, hidden, n_hidden_layers, n_out, n_dof, seed, ctypes.byref(h)))
    return h


def ts_surrogate_free(sur):
    lib().ts_surrogate_free(sur)


def ts_surrogate_num_params(sur) -> int:
    return int(lib().ts_surrogate_num_params(sur))


def ts_surrogate_get_params(sur, out: np.ndarray):
    _check(lib().ts_surrogate_get_params(sur, _fp(out), out.size))
    return out


def ts_surrogate_set_params(sur, flat: np.ndarray):
    _check(lib().ts_surrogate_set_params(sur, _fp(flat), flat.size))


def ts_surrogate_forward(sur, X, B, out, stream=None):
    _check(lib().ts_surrogate_forward(sur, X.data_ptr(), B, out.data_ptr(), _stream_ptr(stream)))
    return out


def ts_surrogate_gradient(sur, X, T, B, grad, stream=None) -> float:
    loss = ctypes.c_double()
    _check(lib().ts_surrogate_gradient(sur, X.data_ptr(), T.data_ptr(), B,
                                       None if grad is None else grad.data_ptr(), ctypes.byref(loss),
                                       _stream_ptr(stream)))
    return loss.value


def ts_surrogate_adam(sur, grad, lr, stream=None):
    _check(lib().ts_surrogate_adam(sur, grad.data_ptr(), lr, _stream_ptr(stream)))


def ts_surrogate_fit_basis(sur, Y, S, stream=None):
    _check(lib().ts_surrogate_fit_basis(sur, Y.data_ptr(), S, _stream_ptr(stream)))


def ts_surrogate_basis_rank(sur, sigma: np.ndarray | None = None) -> int:
    p = None if sigma is None else sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return int(lib().ts_surrogate_basis_rank(sur, p))


def ts_surrogate_coefficients(sur, Y, S, A, stream=None):
    _check(lib().ts_surrogate_coefficients(sur, Y.data_ptr(), S, A.data_ptr(), _stream_ptr(stream)))
    return A


def ts_surrogate_train(sur, X_host: np.ndarray, Y, S, epochs, batch, lr, seed, loss_hist: np.ndarray,
                       stream=None):
    _check(lib().ts_surrogate_train(sur, _fp(X_host), Y.data_ptr(), S, epochs, batch, lr, seed,
                                    loss_hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    _stream_ptr(stream)))
    return loss_hist


def ts_surrogate_guess(sur, prob, x_host: np.ndarray, y, stream=None):
    _check(lib().ts_surrogate_guess(sur, prob, _fp(x_host), y.data_ptr(), _stream_ptr(stream)))
    return y


class Surrogate:
    """POD basis + fully connected network giving a Newton initial guess (ts_surrogate_*)."""

    def __init__(self, n_in, hidden, n_hidden_layers, n_out, n_dof, seed=0):
        self.h = ts_surrogate_create(n_in, hidden, n_hidden_layers, n_out, n_dof, seed)
        self.n_in, self.n_out, self.n_dof = n_in, n_out, n_dof
        self.sizes = [n_in] + [hidden] * n_hidden_layers + [n_out]

    @property
    def n_params(self) -> int:
        return int(lib().ts_surrogate_num_params(self.h))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().ts_surrogate_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(lib().ts_surrogate_set_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def layers(self, flat=None):
        """[(W [out][in], b [out])] views of a flat parameter vector."""
        flat = self.get_params() if flat is None else flat
        out, off = [], 0
        for n_in, n_out in zip(self.sizes[:-1], self.sizes[1:]):
            W = flat[off: off + n_in * n_out].reshape(n_out, n_in)
            off += n_in * n_out
            b = flat[off: off + n_out]
            off += n_out
            out.append((W, b))
        return out

    def forward(self, X, stream=None):
        import torch
        X = X.contiguous()
        out = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        _check(lib().ts_surrogate_forward(self.h, X.data_ptr(), X.shape[0], out.data_ptr(), _stream_ptr(stream)))
        return out

    def gradient(self, X, T, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        _check(lib().ts_surrogate_gradient(self.h, X.contiguous().data_ptr(), T.contiguous().data_ptr(),
                                           X.shape[0], g.data_ptr(), ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value, g

    def adam(self, grad, lr, stream=None):
        _check(lib().ts_surrogate_adam(self.h, grad.data_ptr(), lr, _stream_ptr(stream)))

    def fit_basis(self, Y, stream=None):
        """Y: CUDA float64 [S][n_dof] snapshots."""
        _check(lib().ts_surrogate_fit_basis(self.h, Y.contiguous().data_ptr(), Y.shape[0], _stream_ptr(stream)))
        sig = np.zeros(self.n_out)
        k = lib().ts_surrogate_basis_rank(self.h, sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return sig[:k]

    def coefficients(self, Y, stream=None):
        import torch
        A = torch.empty((Y.shape[0], self.n_out), dtype=torch.float32, device=Y.device)
        _check(lib().ts_surrogate_coefficients(self.h, Y.contiguous().data_ptr(), Y.shape[0], A.data_ptr(),
                                               _stream_ptr(stream)))
        return A

    def train(self, X_host, Y, epochs, batch, lr, seed=0, stream=None):
        X = np.ascontiguousarray(X_host, dtype=np.float32)
        hist = np.zeros(epochs)
        _check(lib().ts_surrogate_train(self.h, X.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        Y.contiguous().data_ptr(), X.shape[0], epochs, batch, lr, seed,
                                        hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream)))
        return hist

    def guess(self, problem, x, y, stream=None):
        """y (CUDA float64 field of ``problem``, a GLSProblem) <- surrogate on its free entries."""
        xx = np.ascontiguousarray(x, dtype=np.float32)
        _check(lib().ts_surrogate_guess(self.h, problem.prob, xx.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        y.data_ptr(), _stream_ptr(stream)))
        return y

    def close(self):
        if getattr(self, "h", None):
            lib().ts_surrogate_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ tracer (eq. 3D-weak)

def ts_tracer_create(mesh, N, kappa, omega, C_I=3.0):
    h = ctypes.c_void_p()
    _check(lib().ts_tracer_create(mesh, N, kappa, omega, C_I, ctypes.byref(h)))
    return h


def ts_tracer_free(tracer):
    lib().ts_tracer_free(tracer)


def ts_tracer_set_dirichlet(tracer, tag):
    _check(lib().ts_tracer_set_dirichlet(tracer, tag))


def ts_tracer_residual(tracer, a, phi, r, stream=None):
    import torch
    for t in (a, phi, r):
        if not t.is_cuda or not t.is_contiguous() or t.dtype != phi.dtype:
            raise ValueError("a, phi, r must be contiguous CUDA tensors of one dtype")
    p = 64 if phi.dtype == torch.float64 else 32
    _check(lib().ts_tracer_residual(tracer, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                    ctypes.c_void_p(r.data_ptr()), p, _stream_ptr(stream)))
    return r


def ts_tracer_set_stabilised(tracer, gls):
    _check(lib().ts_tracer_set_stabilised(tracer, int(gls)))


def ts_tracer_solve(tracer, a, phi, tol=1e-10, krylov=100, max_matvec=20000, stream=None):
    """phi (FP64 CUDA [V, N, 2], Dirichlet values in place) <- root of the tracer residual."""
    import torch
    for t in (a, phi):
        if not t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64:
            raise ValueError("a and phi must be contiguous CUDA float64 tensors")
    nmv, rel = ctypes.c_int(), ctypes.c_double()
    _check(lib().ts_tracer_solve(tracer, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(phi.data_ptr()), tol,
                                 krylov, max_matvec, ctypes.byref(nmv), ctypes.byref(rel), _stream_ptr(stream)))
    return {"matvecs": nmv.value, "rel": rel.value}


class Tracer:
    """Time-spectral GLS convection-diffusion residual of a scalar on a mesh
    (ts_tracer_*); phi and r are CUDA tensors [V, N, 2], the velocity a [V, 3, N, 2]."""

    def __init__(self, mesh_handle, n_nodes, N, kappa, omega, C_I=3.0, dirichlet_tags=()):
        self.h = ts_tracer_create(mesh_handle, N, kappa, omega, C_I)
        self.N, self.n_nodes = N, n_nodes
        for tag in dirichlet_tags:
            ts_tracer_set_dirichlet(self.h, tag)

    def residual(self, a, phi, r=None, stream=None):
        import torch
        return ts_tracer_residual(self.h, a, phi, torch.empty_like(phi) if r is None else r, stream)

    def stabilised(self, gls=True):
        ts_tracer_set_stabilised(self.h, gls)

    def solve(self, a, phi, tol=1e-10, krylov=100, max_matvec=20000, stream=None):
        return ts_tracer_solve(self.h, a, phi, tol, krylov, max_matvec, stream)

    def close(self):
        if getattr(self, "h", None):
            ts_tracer_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
