"""Benchmark of the GB300 time-spectral GLS hot path (one JSON line on rank 0).

Workload: the Fontan-like synthetic cross junction (two inlets of radius
1.0 and 0.8, two outlets of radius 0.9, arm length 6), seeded tetrahedral
mesh of about 188k tets / 38k nodes, N = 7 modes, Re 500, Wo 10, random 1/k^2
inflow waveforms, resistance outlets R = 1.

A step is one pseudo-time Newton-GMRES step of the mixed-precision solver
through the C ABI (``ts_solve``): the FP64 residual of eq. (Rmc) with tau
at every quadrature point, an approximate-diagonal right preconditioner, and
GMRES with a fixed budget of KRYLOV FP32 tangent products (eq. K_mat, tau
frozen, A linearised) and FP64 classical Gram-Schmidt, then the update.
``value`` = element-mode operator evaluations per second, E * N * (tangent
products + residuals) / time.  The time to ||r|| <= 1e-8 r_ref of the full
solve, mixed vs FP64, is measured once beside the timed steps.

``--impl reference`` times the CPU oracle (FP64 numpy, complex modes) on the
host cores on a bounded element sample of the same workload, same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")   # the CPU oracle runs on one core
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np

METRIC = "GLS operator element-mode evals/s; time to 1e-8 residual, mixed vs FP64 on GB300"
KRYLOV = 30
N_MODES = 7
WAVE_AMP = 0.05   # 1/n^2 waveform scale (the configuration fixes the decay, not the amplitude)
SOLVE_OPTS = dict(tol=1e-8, krylov=100, eps_ls=0.05, max_matvec=1000, precond=1, ser=1.0, dt_max=8.0,
                  raise_on_noconv=False)


def _sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload(seed_mesh=1, h=0.123):
    from workloads import cases, meshgen as mg
    mesh = mg.junction(h=h, seed=seed_mesh)
    return cases.junction_case(N=N_MODES, Re=500.0, Wo=10.0, wave_seed=100, resistance=1.0, mesh=mesh,
                               amp=WAVE_AMP)


def _library_inflow(g, case):
    """Inlet data through the library (ts_set_inlet: parabolic profile x the
    inflow waveform's flow-rate coefficients) and the paper's initial guess
    (ts_initial_guess): a new FP64 CUDA field."""
    from workloads import meshgen as mg
    for ax, sg, R, tag in mg.JUNCTION_ARMS:
        if tag not in (mg.TAG_INLET1, mg.TAG_INLET2):
            continue
        # the arm's axis passes through the origin; inflow points along -sg * axis
        direction = np.zeros(3)
        direction[mg._AX[ax]] = -sg
        centre = np.zeros(3)
        centre[mg._AX[ax]] = sg * case.mesh.info.get("arm_len", 6.0)
        Q = np.asarray(case.info["waves"][tag]) * np.pi * R ** 2
        g.set_inlet(tag, Q, "parabolic", centre=centre, direction=direction, radius=R)
    return g.initial_guess()


def _config(case, extra=None):
    c = {"workload": "fontan-like cross junction, P1-P1 tets, time-spectral GLS Navier-Stokes",
         "n_tets": int(case.mesh.n_tets), "n_nodes": int(case.mesh.n_nodes), "n_modes": case.N,
         "Re": 500.0, "Wo": 10.0, "outlets": "resistance R=1", "waveform": f"1/n^2, scale {WAVE_AMP}",
         "step": f"1 pseudo-time Newton step: FP64 residual + {KRYLOV} FP32 tangent products in FP64 GMRES",
         "l2": "inputs larger than L2 (tau cache 0.27 GB, Krylov basis 0.5 GB)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index=0):
        self.samples, self.proc, self.thread = [], None, None
        self.index = index

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])
        self.thread = threading.Thread(target=rd, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx.append(float(s[1]))
                for k, n in enumerate(names):
                    if s[3 + k].lower().startswith("active"):
                        reasons.add(n)
            except Exception:
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _jvp_bytes(case, b=4):
    """Algorithmic bytes of one tangent product (eq. K_mat, LIN_A variant)."""
    V, E, N = case.mesh.n_nodes, case.mesh.n_tets, case.N
    nm = 2 * N - 1
    return (V * 8 * N * b          # v
            + V * 8 * N * b        # linearisation state u0, p0 (LIN_A reads both)
            + V * 8 * N * b        # Hv
            + 16 * E               # connectivity
            + 12 * V               # coordinates (geometry)
            + E * 4 * nm * (nm + 1) // 2 * b   # tau per quadrature point
            + E * 4 * 3 * 2 * N * b)           # tau L(u0) per point (LIN_A)


def _jvp_bytes_model(case, b=4):
    """Algorithmic bytes of one tangent product in the operator's roofline model:
    v and Hv (8N values per node), the linearisation velocity u0 (6N per node),
    connectivity (16 B per element), coordinates (12 B per node) and tau (the
    packed n_m (n_m + 1) / 2 entries at each of the 4 points of every element)."""
    V, E, N = case.mesh.n_nodes, case.mesh.n_tets, case.N
    nm = 2 * N - 1
    return (V * 8 * N * b + V * 6 * N * b + V * 8 * N * b + 16 * E + 12 * V
            + E * 4 * nm * (nm + 1) // 2 * b)


def _jvp_flops(case):
    """Algorithmic flops of one tangent product in the operator's arithmetic
    model at N = 7 (K = 19 time samples): about 6.3k multiply-adds per
    quadrature point (the forward and inverse time-sample transforms of the
    convective products about 4.4k of them) and about 3k per element, i.e.
    2 x (4 x 6300 + 3000) flops per element.  None for other N."""
    if case.N != 7:
        return None
    return 2 * (4 * 6300 + 3000) * case.mesh.n_tets


def _tau_flops(case):
    """Algorithmic flops of tau at every quadrature point (eq. 3D-tau): about
    45 n_m^3 per point -- forming M ~6 n_m^3, a Jacobi eigensolve ~30-40 n_m^3,
    tau = V f(Lambda) V^T ~2 n_m^3 -- with n_m = 2N - 1, 4 points per element."""
    nm = 2 * case.N - 1
    return 4 * case.mesh.n_tets * 45 * nm ** 3


def _tau_dd_instr(case):
    """FP32 instructions of the double-float refinement in one tau_dd launch.

    Per quadrature point (n = 2N - 1, t = n(n+1)/2): M (3 t n), the second
    Newton-Schulz Gram matrix, B and tau (t n each, symmetric) and the four
    full products V H twice, M V, Z V^T (n^3 each) are double-float
    multiply-adds of 15 FP32 instructions; the first Gram matrix (t n) takes
    FP32 factors, 13 instructions.  The FP32 Jacobi sweeps (data-dependent
    count) are not counted."""
    n = 2 * case.N - 1
    t = n * (n + 1) // 2
    per_point = 15 * (6 * t * n + 4 * n ** 3) + 13 * t * n
    return 4 * case.mesh.n_tets * per_point


def _profile_traffic(kernel_src, name="jvp32_traffic.json", key="dram_bytes_per_jvp"):
    """DRAM traffic per launch from a committed ncu summary, if still current."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            d = json.load(f)
        h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
        if d.get("source_sha") == h:
            return float(d[key])
    except Exception:
        pass
    return None


def _dist(backend="nccl"):
    """Process group of a torchrun launch (RANK, WORLD_SIZE, MASTER_* from the
    environment); None on one rank.  Each rank runs its own replica of the
    workload (no data-path collective)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
        return dist, rank, ws
    return None, rank, ws


def _max_over_ranks(dist, x):
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(ws, n_tets, n_modes, ops, seconds):
    """Whole-job element-mode evaluations per second: every rank runs the same
    replica, so the units processed are ws times one rank's."""
    return ws * n_tets * n_modes * ops / seconds


def run_gpu(args):
    import torch

    import paper_2311_09465_gb300 as ts

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    case = _workload()
    E, N = case.mesh.n_tets, case.N
    g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=args.dt)
    stream = torch.cuda.current_stream()
    y0 = _library_inflow(g, case)
    y = y0.clone()
    # every timed step is one residual + KRYLOV products (no step rejection)
    opts = dict(precision=32, tol=1e-300, max_steps=1, krylov=KRYLOV, eps_ls=1e-30,
                max_matvec=KRYLOV, precond=1, raise_on_noconv=False, reject=0.0)
    # warm-up: pseudo-time steps from the plain initial guess
    for _ in range(args.warmup):
        g.solve(y, **opts)
    torch.cuda.synchronize()

    # ---- timed region: K pseudo-time steps in one solve call
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ts.ts_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rep = g.solve(y, **dict(opts, max_steps=args.steps))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = ts.ts_launch_count() - l0
    clk = clocks.stop()
    t_total = ev0.elapsed_time(ev1) / 1e3
    t_total = _max_over_ranks(dist, t_total)
    ops = rep["matvecs"] + rep["steps"] + 1          # tangent products + residuals
    value = _job_rate(ws, E, N, ops, t_total)
    ms_step = t_total / args.steps * 1e3

    # ---- kernel timings.  The dominant kernel of the step (largest share of
    # device time in the ncu launch list) is tau_dd_kernel, the tau of the FP64
    # residual; its time and the tangent product's element kernel come from the
    # library's own CUDA events on the launching stream (ts_stage_times).
    R = 20
    r64 = torch.empty_like(y)
    t_tau, t_res64 = [], []
    for _ in range(3):
        ts.ts_residual(g.prob, y, r64)
        st_ = ts.ts_stage_times(g.prob)
        t_tau.append(st_["tau_ms"] / 1e3)
        t_res64.append(st_["residual_element_ms"] / 1e3)
    t_tau_cold = float(np.mean(t_tau))
    t_res64 = float(np.mean(t_res64))
    # the roofline's launch time: the tau launches of the timed solve (CUDA
    # events around each one, summed by ts_solve; all but the first start
    # their eigensolve from the previous step's eigenvectors)
    t_tau = rep["t_tau"] / max(rep["n_residual"], 1) if rep.get("n_residual") else t_tau_cold
    y32 = y.float().contiguous()
    ts.ts_residual(g.prob, y32, torch.empty_like(y32))
    v32 = torch.tensor(np.random.default_rng(0).standard_normal(y.shape), dtype=torch.float32, device="cuda")
    hv = torch.empty_like(v32)
    for _ in range(3):
        ts.ts_jvp(g.prob, v32, hv)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(R):
        ts.ts_jvp(g.prob, v32, hv)
    e1.record(stream)
    torch.cuda.synchronize()
    t_jvp = e0.elapsed_time(e1) / 1e3 / R
    t_jel = []
    for _ in range(R):
        ts.ts_jvp(g.prob, v32, hv)
        t_jel.append(ts.ts_stage_times(g.prob)["jvp_element_ms"] / 1e3)
    t_jel = float(np.mean(t_jel))
    # residual (tau refresh) in FP32 for the breakdown
    r32 = torch.empty_like(y32)
    e0.record(stream)
    for _ in range(3):
        ts.ts_residual(g.prob, y32, r32)
    e1.record(stream)
    torch.cuda.synchronize()
    t_res32 = e0.elapsed_time(e1) / 1e3 / 3
    # whole FP64 residual (tau + element pass + boundary terms) and plain FP64 products
    e0.record(stream)
    for _ in range(3):
        ts.ts_residual(g.prob, y, r64)
    e1.record(stream)
    torch.cuda.synchronize()
    t_res64_all = e0.elapsed_time(e1) / 1e3 / 3
    v64 = v32.double()
    hv64 = torch.empty_like(v64)
    t_jvp64 = {}
    for elem in ("native", "doublefloat"):
        g.option(element64=elem)
        ts.ts_jvp(g.prob, v64, hv64)
        e0.record(stream)
        for _ in range(5):
            ts.ts_jvp(g.prob, v64, hv64)
        e1.record(stream)
        torch.cuda.synchronize()
        t_jvp64[elem] = e0.elapsed_time(e1) / 1e3 / 5
    peak, peak_kind = _peaks()
    alg = _jvp_bytes_model(case)
    alg_lin_a = _jvp_bytes(case)
    achieved = alg / t_jel / 1e9
    csrc = os.path.join(ROOT, "paper_2311_09465_gb300", "csrc")
    traffic = _profile_traffic(os.path.join(csrc, "jvp32.cuh"))
    # FP32 peaks: SMs x 128 FP32 lanes x the maximum SM clock (instructions), x 2 (FMA flops)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * 128 * _sm_max_mhz() * 1e6 / 1e12
    fma_peak = 2 * alu_peak
    tau_work = _tau_dd_instr(case)
    tau_flops = _tau_flops(case)
    jvp_flops = _jvp_flops(case)
    tau_traffic = _profile_traffic(os.path.join(csrc, "tau_dd.cu"), "tau_dd_traffic.json", "dram_bytes_per_launch")

    # ---- end-to-end through the public API with host buffers
    y_host = y0.cpu().pin_memory()
    y_back = torch.empty_like(y_host).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    yd = y_host.to("cuda", non_blocking=True)
    rep_e = g.solve(yd, **dict(opts, max_steps=args.steps))
    y_back.copy_(yd, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = _max_over_ranks(dist, time.perf_counter() - t0)
    ops_e = rep_e["matvecs"] + rep_e["steps"] + 1
    e2e = {"value": _job_rate(ws, E, N, ops_e, t_e2e), "unit": "element-mode evals/s",
           "h2d_bytes_per_step": int(y_host.numel() * 8 / args.steps),
           "d2h_bytes_per_step": int(y_host.numel() * 8 / args.steps)}

    # ---- time to residual 1e-8 r_ref: mixed vs plain FP64 (same GPU)
    ttr = {}
    if args.solve:
        ttr = _time_to_residual(ts, torch, case, g, args)
    cpu = _cpu_baseline(case, args) if (rank == 0 and ws == 1 and not args.no_cpu) else None
    out = {
        "metric": METRIC, "value": value, "unit": "element-mode evals/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic seeded junction mesh and inflow (patient Fontan data not available)",
        "config": _config(case, {"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}),
        "e2e": e2e, "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": tau_flops / t_tau / 1e12, "peak": fma_peak,
                     "unit": "TFLOP/s", "frac": tau_flops / t_tau / 1e12 / fma_peak,
                     "traffic": tau_traffic,
                     "kernel": "tau_dd_kernel<7> (tau of the FP64 residual, double-float refinement)",
                     "algorithmic_flops": tau_flops, "flop_model": "45 n_m^3 per quadrature point",
                     "launch_ms": t_tau * 1e3, "launches_timed": int(rep.get("n_residual", 0)),
                     "launch_ms_cold": t_tau_cold * 1e3,
                     "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {_sm_max_mhz():.0f} MHz "
                                    "(an FMA probe measured 78.4 TFLOP/s FP32, 1.25 FP64)",
                     "issue": {"achieved": tau_work / t_tau / 1e12, "peak": alu_peak,
                               "unit": "T FP32 instructions/s", "frac": tau_work / t_tau / 1e12 / alu_peak,
                               "instructions": tau_work}},
        "roofline_tangent": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "kernel": "jvp32_kernel<7, LIN_A> (FP32 tangent product, element pass)",
                             "algorithmic_bytes": alg, "launch_ms": t_jel * 1e3,
                             "algorithmic_bytes_with_lin_a_tau_L": alg_lin_a,
                             "frac_with_lin_a_tau_L": alg_lin_a / t_jel / 1e9 / peak,
                             "product_ms": t_jvp * 1e3, "peak_source": peak_kind,
                             "alu": None if jvp_flops is None else {
                                 "achieved": jvp_flops / t_jel / 1e12, "peak": fma_peak, "unit": "TFLOP/s",
                                 "frac": jvp_flops / t_jel / 1e12 / fma_peak, "flops": jvp_flops,
                                 "flop_model": "2 x (4 x 6300 + 3000) per element at N = 7",
                                 "peak_source": "derived FP32 FMA peak, as roofline.peak"}},
        "operator_throughput": {
            "unit": "element-mode evals/s",
            "residual_fp64": E * N / t_res64_all, "residual_fp32": E * N / t_res32,
            "jvp_fp32": E * N / t_jvp, "jvp_fp64": E * N / t_jvp64["native"],
            "jvp_fp64_doublefloat": E * N / t_jvp64["doublefloat"],
            "ms": {"residual_fp64": t_res64_all * 1e3, "residual_fp32": t_res32 * 1e3,
                   "jvp_fp32": t_jvp * 1e3, "jvp_fp64": t_jvp64["native"] * 1e3,
                   "jvp_fp64_doublefloat": t_jvp64["doublefloat"] * 1e3}},
        "cpu_baseline": cpu,
        "clocks": clk,
        "breakdown": {"jvp_fp32_ms": t_jvp * 1e3, "jvp_element_kernel_ms": t_jel * 1e3,
                      "tau_dd_ms": t_tau * 1e3, "residual_fp64_element_pass_ms": t_res64 * 1e3,
                      "residual_fp32_ms": t_res32 * 1e3,
                      "solve_report": {k: rep[k] for k in ("steps", "matvecs", "t_residual", "t_jvp", "t_krylov")}},
        "time_to_residual_1e-8": ttr or None,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()


def _elem64(tau64):
    """The plain FP64 legs run every FP64 operation as FP64 instructions
    (tau by the FP64 refinement, the native FP64 element operator); the mixed
    legs use the library defaults (double-float tau and element pass)."""
    return "native" if tau64 == "refine" else None


def _one_solve(ts, torch, g, y0, prec, max_steps):
    yy = torch.tensor(y0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rs = g.solve(yy, precision=prec, max_steps=max_steps, **SOLVE_OPTS)
    torch.cuda.synchronize()
    return yy, {"seconds": time.perf_counter() - t0, "converged": rs["status"] == 0,
                "r_final": rs["r_final"], "steps": rs["steps"], "matvecs": rs["matvecs"],
                "t_residual": rs["t_residual"], "t_jvp": rs["t_jvp"], "t_krylov": rs["t_krylov"]}


def _time_to_residual(ts, torch, case, g, args):
    """Full solves from the paper's initial guess to ||r|| <= 1e-8 r_ref."""
    from workloads import cases, meshgen as mg
    out = {}
    # the Womersley pipe (R 1, L 5, ~9.6k tets), N = 3, Re 100, Wo 5
    pipe = cases.pipe_case(N=3, Re=100.0, Wo=5.0, mesh=mg.pipe(nc=4, nr=4, nz=20))
    res = {}
    # mixed: FP32 tangent products, FP64 GMRES, outer residual with double-float tau;
    # plain FP64: FP64 products and the FP64 tau refinement
    for prec, tau64 in ((32, "doublefloat"), (64, "refine")):
        gp = ts.GLSProblem(pipe, variant="lin_a", dt_pseudo=0.5, tau64=tau64, element64=_elem64(tau64))
        yy, rep = _one_solve(ts, torch, gp, pipe.y0, prec, 60)
        rep["tau64"] = tau64
        res["mixed" if prec == 32 else "fp64"] = rep
        if prec == 32:
            y_mixed = yy
        gp.close()
    if res["mixed"]["converged"] and res["fp64"]["converged"]:
        res["speedup_mixed_over_fp64"] = res["fp64"]["seconds"] / res["mixed"]["seconds"]
        res["field_rel_l2_mixed_vs_fp64"] = float((y_mixed - yy).norm() / yy.norm())
    res["workload"] = f"pipe, {pipe.mesh.n_tets} tets, N=3, Re 100, Wo 5"
    out["pipe"] = res
    out["batched"] = _batched_ttr(ts, torch)
    out["surrogate"] = _surrogate_ttr(ts, torch)
    out["junction"] = _junction_ttr(ts, torch, case, args)
    return out


JUNCTION_SOLVE = dict(tol=1e-8, max_steps=120, krylov=100, eps_ls=0.05, max_matvec=1000, precond=3, ser=1.0,
                      dt_max=2.0, reject=4.0, raise_on_noconv=False)


def _junction_ttr(ts, torch, case, args):
    """Time to ||r|| <= 1e-8 r_ref on the bench junction (188k tets, N = 7, Wo 10,
    resistance outlets) at the largest Re this solver converges from the paper's
    initial guess, Re 100: mixed precision (FP32 LIN_A products, FP64 GMRES and
    outer residual) always; plain FP64 (FP64 products and tau refinement) with
    --junction-fp64 (about 15 minutes on one GB300).  The inflow is set through
    ts_set_inlet; r_ref is the norm at the initial guess."""
    from workloads import cases
    jc = cases.junction_case(N=case.N, Re=args.junction_re, Wo=10.0, wave_seed=100, resistance=1.0,
                             mesh=case.mesh, amp=WAVE_AMP)
    res = {"workload": f"junction {jc.mesh.n_tets} tets, N={jc.N}, Re {args.junction_re}, Wo 10, resistance R=1",
           "solver": {k: v for k, v in JUNCTION_SOLVE.items() if k != "raise_on_noconv"}}
    legs = [("mixed", 32, "doublefloat")] + ([("fp64", 64, "refine")] if args.junction_fp64 else [])
    fields = {}
    for name, prec, tau64 in legs:
        g = ts.GLSProblem(jc, variant="lin_a", dt_pseudo=0.2, tau64=tau64, element64=_elem64(tau64))
        y = _library_inflow(g, jc)
        r_ref = float(g.residual(y).norm())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = g.solve(y, precision=prec, r_ref=r_ref, **JUNCTION_SOLVE)
        torch.cuda.synchronize()
        res[name] = {"seconds": time.perf_counter() - t0, "converged": rep["status"] == 0, "r_final": rep["r_final"],
                     "steps": rep["steps"], "matvecs": rep["matvecs"], "t_residual": rep["t_residual"],
                     "t_jvp": rep["t_jvp"], "t_krylov": rep["t_krylov"], "t_precond": rep["t_precond"],
                     "tau64": tau64}
        fields[name] = y
        g.close()
    if "fp64" in fields and res["mixed"]["converged"] and res["fp64"]["converged"]:
        res["speedup_mixed_over_fp64"] = res["fp64"]["seconds"] / res["mixed"]["seconds"]
        res["field_rel_l2_mixed_vs_fp64"] = float((fields["mixed"] - fields["fp64"]).norm() / fields["fp64"].norm())
    return res


def _pipe_family(rng, n, meshes):
    """Seeded pulsatile pipe instances: uneven meshes, N in {3, 5, 7}, Re ~ U(60, 140)."""
    from workloads import cases
    out = []
    for i in range(n):
        N = (3, 5, 7)[i % 3]
        Re = float(rng.uniform(60.0, 140.0))
        U = cases.waveform_random(N, int(rng.integers(0, 2**31)), amp=0.4)
        out.append((cases.pipe_case(N=N, Re=Re, Wo=5.0, amps=tuple(U), mesh=meshes[i % len(meshes)]), U, Re))
    return out


def _batched_ttr(ts, torch):
    """Lockstep batched mixed solve vs the same instances one by one (mixed and plain FP64)."""
    from workloads import meshgen as mg
    meshes = [mg.pipe(nc=3, nr=2, nz=8), mg.pipe(nc=2, nr=2, nz=10), mg.pipe(nc=4, nr=3, nz=12),
              mg.pipe(nc=3, nr=2, nz=16)]
    inst = _pipe_family(np.random.default_rng(1000), 8, meshes)
    opts = dict(tol=1e-8, max_steps=60, krylov=60, eps_ls=0.05, ser=1.0, dt_max=8.0, raise_on_noconv=False)
    res = {"workload": f"{len(inst)} pipe instances, {sorted(set(m.n_tets for m in meshes))} tets, "
                       "N in {3,5,7}, Re U(60,140), Wo 5, own 1/n^2 waveforms"}
    seq = {}
    for prec, tau64 in ((32, "doublefloat"), (64, "refine")):
        t, ok, fields = 0.0, True, []
        for c, _, _ in inst:
            g = ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.5, tau64=tau64, element64=_elem64(tau64))
            y = torch.tensor(c.y0, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = g.solve(y, precision=prec, **opts)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            ok = ok and rep["status"] == 0
            fields.append(y)
            g.close()
        seq["mixed" if prec == 32 else "fp64"] = (t, ok, fields)
    gs = [ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.5) for c, _, _ in inst]
    ys = [torch.tensor(c.y0, dtype=torch.float64, device="cuda") for c, _, _ in inst]
    b = ts.Batch(gs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = b.solve(ys, **opts)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    res["batched_seconds"] = tb
    res["batched_converged"] = all(r["status"] == 0 for r in reps)
    res["launch_shape"] = b.launch_shape()
    res["sequential_mixed_seconds"], res["sequential_mixed_converged"] = seq["mixed"][0], seq["mixed"][1]
    res["sequential_fp64_seconds"], res["sequential_fp64_converged"] = seq["fp64"][0], seq["fp64"][1]
    res["speedup_over_sequential_fp64"] = seq["fp64"][0] / tb
    res["speedup_over_sequential_mixed"] = seq["mixed"][0] / tb
    res["max_field_rel_l2_vs_sequential_fp64"] = max(
        float((y - f).norm() / f.norm()) for y, f in zip(ys, seq["fp64"][2]))
    b.close()
    for g in gs:
        g.close()
    return res


def _surrogate_ttr(ts, torch, n_train=32, n_test=4):
    """Train the learned initial guess on solves of the method, then time held-out solves."""
    from workloads import cases, meshgen as mg
    mesh = mg.pipe(nc=3, nr=2, nz=10)
    rng = np.random.default_rng(2000)
    opts = dict(tol=1e-8, max_steps=60, krylov=60, eps_ls=0.05, ser=1.0, dt_max=8.0, raise_on_noconv=False)

    def sample():
        Re = float(rng.uniform(60.0, 140.0))
        U = cases.waveform_random(3, int(rng.integers(0, 2**31)), amp=0.4)
        return cases.pipe_case(N=3, Re=Re, Wo=5.0, amps=tuple(U), mesh=mesh), U, Re

    X, Y = [], []
    t0 = time.perf_counter()
    for _ in range(n_train):
        c, U, Re = sample()
        g = ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.5)
        y = torch.tensor(c.y0, dtype=torch.float64, device="cuda")
        g.solve(y, precision=32, **opts)
        X.append(cases.surrogate_inputs([U], Re, 5.0, harmonics=2))
        Y.append(y.reshape(-1))
        g.close()
    Yd = torch.stack(Y)
    s = ts.Surrogate(len(X[0]), 128, 3, 16, Yd.shape[1], seed=7)
    s.fit_basis(Yd)
    hist = s.train(np.array(X), Yd, epochs=400, batch=16, lr=2e-3, seed=8)
    t_train = time.perf_counter() - t0
    rows = []
    for _ in range(n_test):
        c, U, Re = sample()
        x = cases.surrogate_inputs([U], Re, 5.0, harmonics=2)
        row = {}
        for name, prec, tau64, guess in (("fp64_plain", 64, "refine", False), ("mixed_plain", 32, "doublefloat", False),
                                          ("mixed_surrogate", 32, "doublefloat", True)):
            g = ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.5, tau64=tau64, element64=_elem64(tau64))
            y = torch.tensor(c.y0, dtype=torch.float64, device="cuda")
            r_ref = float(g.residual(y).norm())
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if guess:
                s.guess(g, x, y)
            rep = g.solve(y, precision=prec, r_ref=r_ref, **opts)
            torch.cuda.synchronize()
            row[name] = {"seconds": time.perf_counter() - t1, "steps": rep["steps"], "matvecs": rep["matvecs"],
                         "converged": rep["status"] == 0}
            g.close()
        rows.append(row)
    s.close()
    agg = {k: {"seconds": sum(r[k]["seconds"] for r in rows), "steps": sum(r[k]["steps"] for r in rows),
               "converged": all(r[k]["converged"] for r in rows)} for k in rows[0]}
    return {"workload": f"pipe {mesh.n_tets} tets, N=3, Re U(60,140), Wo 5; {n_train} training solves, "
                        f"{n_test} held out; network 6-128x3-16 (tanh), POD rank <= 16",
            "train_seconds": t_train, "train_loss_first_last": [float(hist[0]), float(hist[-1])],
            "held_out": agg,
            "speedup_surrogate_over_fp64_plain": agg["fp64_plain"]["seconds"] / agg["mixed_surrogate"]["seconds"],
            "speedup_surrogate_over_mixed_plain": agg["mixed_plain"]["seconds"] / agg["mixed_surrogate"]["seconds"]}


def run_surrogate_junction(args, n_train=130, n_test=8, h=0.4, N=7, hidden=512, n_out=128):
    """The learned initial guess at the junction configuration's shape: inputs
    the 16 inflow coefficients (2 inlets x harmonics 1..4 x Re/Im) plus Re and
    Wo, 3 hidden tanh layers of 512, 128 POD coefficients; trained by the
    library's kernels on junction solves of the method (Re ~ U(60, 140), the
    range this solver converges from the plain guess, Wo 10, own 1/n^2 inflow
    per inlet); held-out solves to 1e-8 r_ref from the plain and the learned
    guess (one JSON line).  The training fields are converged to 1e-6 r_ref."""
    import torch

    import paper_2311_09465_gb300 as ts
    from workloads import cases, meshgen as mg

    mesh = mg.junction(h=h, seed=1)
    rng = np.random.default_rng(5000)
    opts = dict(tol=1e-8, max_steps=100, krylov=100, eps_ls=0.05, max_matvec=1000, precond=3, ser=1.0,
                dt_max=2.0, raise_on_noconv=False)

    def sample():
        Re = float(rng.uniform(60.0, 140.0))
        seed = int(rng.integers(0, 2 ** 31))
        c = cases.junction_case(N=N, Re=Re, Wo=10.0, wave_seed=seed, resistance=1.0, mesh=mesh, amp=0.2)
        x = cases.surrogate_inputs([c.info["waves"][mg.TAG_INLET1], c.info["waves"][mg.TAG_INLET2]], Re, 10.0)
        return c, x, Re

    X, Y = [], []
    t0 = time.perf_counter()
    n_conv = 0
    for _ in range(n_train):
        c, x, Re = sample()
        g = ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.2)
        y = _library_inflow(g, c)
        rep = g.solve(y, precision=32, **dict(opts, tol=1e-6))   # training data: 1e-6 r_ref
        n_conv += rep["status"] == 0
        X.append(x)
        Y.append(y.reshape(-1))
        g.close()
    t_solves = time.perf_counter() - t0
    Yd = torch.stack(Y)
    sur = ts.Surrogate(len(X[0]), hidden, 3, n_out, Yd.shape[1], seed=7)
    sigma = sur.fit_basis(Yd)
    hist = sur.train(np.array(X), Yd, epochs=4000, batch=32, lr=1e-3, seed=8)
    t_train = time.perf_counter() - t0 - t_solves
    rows = []
    for _ in range(n_test):
        c, x, Re = sample()
        row = {}
        for name, guess in (("plain", False), ("learned", True)):
            g = ts.GLSProblem(c, variant="lin_a", dt_pseudo=0.2)
            y = _library_inflow(g, c)
            r_ref = float(g.residual(y).norm())
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if guess:
                sur.guess(g, x, y)
            r0 = float(g.residual(y).norm()) / r_ref
            rep = g.solve(y, precision=32, r_ref=r_ref, **opts)
            torch.cuda.synchronize()
            row[name] = {"seconds": time.perf_counter() - t1, "steps": rep["steps"], "matvecs": rep["matvecs"],
                         "converged": rep["status"] == 0, "r0_over_r_ref": r0}
            if guess:
                row["field"] = y
            else:
                y_plain = y
            g.close()
        row["field_rel_l2_learned_vs_plain"] = float((row.pop("field") - y_plain).norm() / y_plain.norm())
        rows.append(row)
    sur.close()
    agg = {k: {"seconds": sum(r[k]["seconds"] for r in rows), "steps": sum(r[k]["steps"] for r in rows),
               "matvecs": sum(r[k]["matvecs"] for r in rows),
               "converged": all(r[k]["converged"] for r in rows)} for k in ("plain", "learned")}
    out = {"surrogate": "junction", "workload": f"junction {mesh.n_tets} tets, N={N}, Re U(60,140), Wo 10, "
                                                 f"1/n^2 inflow x 0.2 per inlet",
           "network": f"{len(X[0])}-{hidden}x3-{n_out} tanh", "train_solves": n_train,
           "train_solves_converged": int(n_conv), "pod_rank": int(len(sigma)), "held_out": n_test,
           "solve_seconds": t_solves, "train_seconds": t_train,
           "train_loss_first_last": [float(hist[0]), float(hist[-1])], "held_out_totals": agg,
           "speedup_learned_over_plain": agg["plain"]["seconds"] / agg["learned"]["seconds"],
           "max_field_rel_l2_learned_vs_plain": max(r["field_rel_l2_learned_vs_plain"] for r in rows),
           "mean_r0_over_r_ref_learned": float(np.mean([r["learned"]["r0_over_r_ref"] for r in rows]))}
    print(json.dumps(out), flush=True)
    return out


def _oracle_step_rate(case, n_elem, n_jvp, seed=0):
    """Oracle residual + tangent products on a fixed element sample; returns (evals/s, seconds)."""
    from oracle import operator as op
    prob = op.problem_from_case(case)
    rng = np.random.default_rng(seed)
    el = np.sort(rng.choice(case.mesh.n_tets, size=n_elem, replace=False))
    y = case.y0
    v = np.random.default_rng(seed + 1).standard_normal(y.shape)
    t0 = time.perf_counter()
    lin = op.linearize(prob, y, elems=el)
    op.apply(prob, lin, y, "frozen")
    for _ in range(n_jvp):
        op.apply(prob, lin, v, "lin_a", mask_dirichlet_input=True)
    dt = time.perf_counter() - t0
    return n_elem * case.N * (n_jvp + 1) / dt, dt


def _cpu_baseline(case, args):
    n_elem = args.cpu_sample
    rate, dt = _oracle_step_rate(case, n_elem, KRYLOV)
    return {"value": rate, "unit": "element-mode evals/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_elem} random elements of the same mesh, 1 residual + {KRYLOV} tangent "
                      f"products (FP64 numpy, complex modes, explicit convolution matrices, "
                      f"library eigensolver); {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    case = _workload()
    rates = []
    for k in range(args.warmup + args.steps):
        rate, dt = _oracle_step_rate(case, args.ref_sample, KRYLOV, seed=k)
        if k >= args.warmup:
            rates.append((rate, dt))
    t = sum(d for _, d in rates)
    work = sum(r * d for r, d in rates)
    value = work / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "element-mode evals/s",
           "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(case),
           "cpu_baseline": {"value": value, "unit": "element-mode evals/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.ref_sample} random elements per step, 1 residual + "
                                      f"{KRYLOV} tangent products"},
           "e2e": {"value": value, "unit": "element-mode evals/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """Mode sweep on the bench junction (N = 3, 7, 15; one JSON line).

    Per N: device time of the FP32 tangent product (the single-launch kernel
    for N <= 7, the colour-ordered one for N = 15) and of the FP64 residual,
    element-mode evaluations per second and achieved GB/s of the product
    (algorithmic bytes as in the bench line), and the relative L2 error of each
    Fourier mode n of the FP32 product and of the FP32 and FP64 residuals
    against the FP64 oracle, over seeded sample nodes whose rows the oracle
    computes exactly from the elements that touch them."""
    import torch

    import paper_2311_09465_gb300 as ts
    from oracle import operator as op
    from workloads import cases, meshgen as mg

    mesh = mg.junction(h=0.123, seed=1)
    rng = np.random.default_rng(23)
    nodes = np.unique(np.concatenate([rng.choice(mesh.n_nodes, 24, replace=False)] + [
        rng.choice(np.nonzero(cases.nodes_with_tag(mesh, t))[0], 3, replace=False)
        for t in (mg.TAG_WALL, mg.TAG_INLET1, mg.TAG_OUTLET1)]))
    peak, peak_kind = _peaks()
    out = []
    for N in (3, 7, 15):
        case = cases.junction_case(N=N, Re=500.0, Wo=10.0, wave_seed=100, resistance=1.0, mesh=mesh,
                                   amp=WAVE_AMP)
        y = case.y0 + 0.3 * cases.random_state(mesh, N, seed=21)
        y[case.dirichlet_mask, 0:3] = case.y0[case.dirichlet_mask, 0:3]
        y[:, :, 0, 1] = 0.0
        v = cases.random_state(mesh, N, seed=22, smooth=False)
        prob = op.problem_from_case(case)
        lin = op.linearize(prob, y, elems=op.element_sample_for_nodes(prob, nodes))
        r_ref = op.apply(prob, lin, y, "frozen")[nodes]
        mc = case.c1 * case.rho / args.dt
        hv_ref = op.apply(prob, lin, v, "lin_a", mask_dirichlet_input=True, mass_coef=mc)[nodes]
        g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=args.dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        y64 = torch.tensor(y, dtype=torch.float64, device="cuda")
        r64 = g.residual(y64)
        e0.record()
        for _ in range(2):
            r64 = g.residual(y64)
        e1.record()
        torch.cuda.synchronize()
        t_res64 = e0.elapsed_time(e1) / 2e3
        r64 = r64.cpu().numpy()[nodes]
        r32 = g.residual(y64.float()).cpu().double().numpy()[nodes]
        v32 = torch.tensor(v, dtype=torch.float32, device="cuda")
        hv = g.jvp(v32)
        e0.record()
        for _ in range(10):
            hv = g.jvp(v32)
        e1.record()
        torch.cuda.synchronize()
        t_jvp = e0.elapsed_time(e1) / 1e4
        hv = hv.cpu().double().numpy()[nodes]

        def per_mode(got, ref):
            errs = []
            for n in range(N):
                d = got[:, :, n, :] - ref[:, :, n, :]
                errs.append(float(np.linalg.norm(d) / max(np.linalg.norm(ref[:, :, n, :]), 1e-300)))
            return errs

        byts = _jvp_bytes(case)
        out.append({"N": N, "K": 3 * N - 2,
                    "tangent_fp32_ms": t_jvp * 1e3, "tangent_element_mode_evals_per_s": case.mesh.n_tets * N / t_jvp,
                    "tangent_gbs": byts / t_jvp / 1e9, "tangent_frac_of_hbm": byts / t_jvp / 1e9 / peak,
                    "residual_fp64_ms": t_res64 * 1e3,
                    "rel_l2_per_mode_tangent_fp32": per_mode(hv, hv_ref),
                    "rel_l2_per_mode_residual_fp32": per_mode(r32, r_ref),
                    "rel_l2_per_mode_residual_fp64": per_mode(r64, r_ref)})
        g.close()
    print(json.dumps({"sweep": "modes", "workload": f"junction {mesh.n_tets} tets, Re 500, Wo 10",
                      "sample_nodes": int(nodes.size), "peak_gbs": peak, "peak_source": peak_kind,
                      "rows": out}), flush=True)


def _spectral_l2(y, n_modes=None):
    """Space-time L2 norm of a modal field [V, 4, N, 2] over the period (Parseval:
    |f|^2 = |f_0|^2 + 2 sum_{n>=1} |f_n|^2), velocity fields only."""
    u = y[:, 0:3]
    w = np.full(u.shape[2], 2.0)
    w[0] = 1.0
    return float(np.sqrt(np.sum(w[None, None, :, None] * u ** 2)))


def mode_error(y_N, y_ref):
    """Relative space-time L2 error of an N-mode field against a reference with
    more modes (the missing modes count as error)."""
    N = y_N.shape[2]
    d = y_ref.copy()
    d[:, :, :N] -= y_N
    return _spectral_l2(d) / _spectral_l2(y_ref)


def run_mode_study(args, Ns=(2, 3, 5, 7, 10), N_ref=15, h=0.3, Re=100.0, Wo=10.0, amp=0.4):
    """Solution error against the number of modes, on the junction with a
    waveform rich in harmonics: every solve iterates to 1e-10 r_ref (mixed
    precision, block Gauss-Seidel preconditioner); the N-mode fields are
    compared with the N_ref-mode field (space-time L2 of the velocity, the
    missing modes counted as error), beside the truncation error of the inflow
    waveform itself (one JSON line)."""
    import torch

    import paper_2311_09465_gb300 as ts
    from workloads import cases, meshgen as mg

    mesh = mg.junction(h=h, seed=1)
    waves = {tag: cases.waveform_random(N_ref, 300 + k, amp=amp) for k, tag in enumerate((mg.TAG_INLET1,
                                                                                         mg.TAG_INLET2))}
    fields, rows = {}, []
    for N in tuple(Ns) + (N_ref,):
        case = cases.junction_case(N=N, Re=Re, Wo=Wo, wave_seed=300, resistance=1.0, mesh=mesh, amp=amp)
        case.info["waves"] = {tag: w[:N] for tag, w in waves.items()}
        g = ts.GLSProblem(case, variant="lin_a", dt_pseudo=0.2)
        y = _library_inflow(g, case)
        r_ref = float(g.residual(y).norm())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = g.solve(y, precision=32, tol=1e-10, r_ref=r_ref, max_steps=150, krylov=100, eps_ls=0.05,
                      max_matvec=2000, precond=3, ser=1.0, dt_max=8.0, raise_on_noconv=False)
        torch.cuda.synchronize()
        fields[N] = y.cpu().numpy()
        rows.append({"N": N, "seconds": time.perf_counter() - t0, "steps": rep["steps"],
                     "matvecs": rep["matvecs"], "r_final": rep["r_final"], "converged": rep["status"] == 0})
        g.close()
    ref = fields[N_ref]
    wref = np.concatenate([w for w in waves.values()])
    wnorm = np.sqrt(sum(abs(w[0]) ** 2 + 2 * np.sum(np.abs(w[1:]) ** 2) for w in waves.values()))
    for row in rows:
        N = row["N"]
        row["field_rel_l2_vs_ref"] = mode_error(fields[N], ref) if N != N_ref else 0.0
        row["inflow_truncation_rel_l2"] = float(np.sqrt(sum(2 * np.sum(np.abs(w[N:]) ** 2)
                                                            for w in waves.values())) / wnorm)
    out = {"study": "mode count", "workload": f"junction {mesh.n_tets} tets, Re {Re}, Wo {Wo}, "
           f"inflow 1/n^2 x {amp} to harmonic {N_ref - 1}", "reference_N": N_ref, "rows": rows}
    if args is not None:
        print(json.dumps(out), flush=True)
    return out


def run_assembled(args, R=20):
    """The assembled block-structured tangent of the paper's variant (section
    2.5.2) on the bench junction: assembly time, storage, the SpMV against
    the matrix-free product of the same variant, and the block preconditioners
    built on it (set-up and application; CUDA events, one JSON line).
    HBM roofline of the SpMV: the records, their column ids and row offsets,
    x and Hv once each, against the measured copy bandwidth."""
    import torch

    import paper_2311_09465_gb300 as ts

    case = _workload()
    g = ts.GLSProblem(case, variant="paper", dt_pseudo=args.dt)
    y = _library_inflow(g, case)
    g.residual(y)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    g.assemble()
    ev[0].record()
    g.assemble()
    ev[1].record()
    torch.cuda.synchronize()
    t_asm = ev[0].elapsed_time(ev[1]) / 1e3
    v = torch.tensor(np.random.default_rng(0).standard_normal(y.shape), dtype=torch.float32, device="cuda")
    hv, hm = torch.empty_like(v), torch.empty_like(v)
    for _ in range(3):
        g.spmv(v, hv)
        g.jvp(v, hm)
    ev[0].record()
    for _ in range(R):
        g.spmv(v, hv)
    ev[1].record()
    torch.cuda.synchronize()
    t_spmv = ev[0].elapsed_time(ev[1]) / 1e3 / R
    ev[0].record()
    for _ in range(R):
        g.jvp(v, hm)
    ev[1].record()
    torch.cuda.synchronize()
    t_mf = ev[0].elapsed_time(ev[1]) / 1e3 / R
    nnz = ts.ts_mesh_connections(g.mesh)
    rec = g.assembled_bytes()
    V, N, E = case.mesh.n_nodes, case.N, case.mesh.n_tets
    alg = rec + 4 * nnz + 4 * (V + 1) + 2 * V * 8 * N * 4
    peak, peak_kind = _peaks()
    # the block preconditioners on their own: set-up and one application
    # (x: an FP64 field; Gauss-Seidel: forward + backward colour sweeps)
    x64 = v.double()
    z64 = torch.empty_like(x64)
    prec = {}
    for kind, name in ((2, "block_jacobi"), (3, "block_gauss_seidel")):
        g.precond_setup(kind)
        ev[0].record()
        g.precond_setup(kind)
        ev[1].record()
        torch.cuda.synchronize()
        t_set = ev[0].elapsed_time(ev[1]) / 1e3
        for _ in range(3):
            g.precond_apply(kind, x64, z64)
        ev[0].record()
        for _ in range(R):
            g.precond_apply(kind, x64, z64)
        ev[1].record()
        torch.cuda.synchronize()
        prec[name] = {"setup_ms": t_set * 1e3, "apply_ms": ev[0].elapsed_time(ev[1]) / R}
    # one Gauss-Seidel sweep reads every off-diagonal record with its column
    # id, the row offsets, the inverted blocks and r once, and writes z once;
    # the application is two sweeps plus the FP64 <-> FP32 conversions
    nf = V * 8 * N
    nb2 = (8 * N) ** 2 * 4
    sweep = (nnz - V) * (rec // nnz) + 4 * nnz + 4 * (V + 1) + V * nb2 + 2 * 4 * nf
    alg_sgs = 2 * sweep + (8 + 4) * nf + 4 * nf + (4 + 8) * nf
    t_sgs = prec["block_gauss_seidel"]["apply_ms"] / 1e3
    prec["block_gauss_seidel"]["roofline"] = {
        "bound": "hbm", "achieved": alg_sgs / t_sgs / 1e9, "peak": peak, "unit": "GB/s",
        "frac": alg_sgs / t_sgs / 1e9 / peak, "algorithmic_bytes": alg_sgs, "peak_source": peak_kind,
        "colours": ts.ts_mesh_node_colours(g.mesh)}
    out = {"assembled": "paper-variant tangent, block-structured (section 2.5.2)",
           "workload": f"junction {E} tets, N={N}", "connections": nnz, "record_bytes": rec,
           "assembly_ms": t_asm * 1e3, "spmv_ms": t_spmv * 1e3, "matrix_free_paper_ms": t_mf * 1e3,
           "spmv_element_mode_evals_per_s": E * N / t_spmv,
           "rel_l2_spmv_vs_matrix_free": float((hv - hm).norm() / hm.norm()),
           "preconditioners": prec,
           "roofline": {"bound": "hbm", "achieved": alg / t_spmv / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": alg / t_spmv / 1e9 / peak, "algorithmic_bytes": alg, "peak_source": peak_kind}}
    print(json.dumps(out), flush=True)
    g.close()


def run_junction_ttr(args):
    """Only the junction time-to-1e-8 leg (its own JSON line)."""
    import torch

    import paper_2311_09465_gb300 as ts
    case = _workload()
    out = _junction_ttr(ts, torch, case, args)
    print(json.dumps({"time_to_residual_1e-8": {"junction": out}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gls", choices=["gls", "reference"])
    ap.add_argument("--dt", type=float, default=0.2, help="pseudo-time step")
    ap.add_argument("--no-solve", dest="solve", action="store_false")
    ap.add_argument("--junction-re", type=float, default=100.0,
                    help="Reynolds number of the junction time-to-1e-8 solve")
    ap.add_argument("--junction-fp64", action="store_true",
                    help="also time the plain FP64 junction solve (about 15 minutes)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=400)
    ap.add_argument("--ref-sample", type=int, default=200)
    ap.add_argument("--junction-ttr", action="store_true",
                    help="only the junction time-to-1e-8 leg (its own JSON line; with --junction-fp64 both legs)")
    ap.add_argument("--surrogate-junction", action="store_true",
                    help="learned initial guess at the junction configuration's network shape (its own JSON line)")
    ap.add_argument("--assembled", action="store_true",
                    help="assembled paper-variant tangent and its SpMV on the junction (its own JSON line)")
    ap.add_argument("--mode-study", action="store_true",
                    help="solution error vs number of modes against a 15-mode reference (its own JSON line)")
    ap.add_argument("--sweep", action="store_true",
                    help="mode sweep N = 3, 7, 15 on the junction (its own JSON line) instead of the bench")
    args = ap.parse_args()
    if args.junction_ttr:
        run_junction_ttr(args)
    elif args.surrogate_junction:
        run_surrogate_junction(args)
    elif args.assembled:
        run_assembled(args)
    elif args.mode_study:
        run_mode_study(args)
    elif args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
