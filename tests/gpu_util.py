"""Helpers shared by the GPU parity tests (not a test module)."""
import math

import numpy as np

from oracle import operator as op


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(y, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(y), dtype=dtype, device="cuda")


def to_np(t):
    return t.detach().double().cpu().numpy()


def mass_coef(case, dt):
    return 0.0 if math.isinf(dt) else case.c1 * case.rho / dt


def oracle_problem(case):
    return op.problem_from_case(case)
