"""The algorithmic models behind the bench line's roofline entries, pinned to
the figures quoted in the design notes and the ncu summaries (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class _Mesh:
    def __init__(self, n_tets, n_nodes):
        self.n_tets, self.n_nodes = n_tets, n_nodes


class _Case:
    def __init__(self, N, n_tets, n_nodes):
        self.N, self.mesh = N, _Mesh(n_tets, n_nodes)


def test_tangent_bytes_at_the_junction():
    import bench
    # v, u0/p0 and Hv (8N values per node, FP32), connectivity, coordinates,
    # packed tau (4 points x 91 entries) and tau L (4 x 3 x 14) per element
    c = _Case(7, 187_989, 38_250)
    V, E = 38_250, 187_989
    expect = 3 * V * 56 * 4 + 16 * E + 12 * V + E * 4 * 91 * 4 + E * 4 * 3 * 14 * 4
    assert bench._jvp_bytes(c) == expect == 429_211_416


def test_tangent_roofline_bytes_model_at_the_junction():
    import bench
    # v, Hv (8N per node), u0 velocity (6N per node), connectivity, coordinates,
    # packed tau (4 points x 91 entries): 300.7 MB at the 188k-tet junction
    V, E = 38_250, 187_989
    expect = V * 56 * 4 + V * 42 * 4 + V * 56 * 4 + 16 * E + 12 * V + E * 4 * 91 * 4
    assert bench._jvp_bytes_model(_Case(7, E, V)) == expect == 300_740_808


def test_tau_flop_model():
    import bench
    # 45 n_m^3 flops per quadrature point, n_m = 2N - 1, 4 points per element
    assert bench._tau_flops(_Case(7, 187_989, 38_250)) == 4 * 187_989 * 45 * 13 ** 3
    assert abs(bench._tau_flops(_Case(7, 187_989, 38_250)) - 7.44e10) < 0.01e10
    assert bench._tau_flops(_Case(1, 3, 4)) == 4 * 3 * 45


def test_jvp_flop_model():
    import bench
    # 6.3k multiply-adds per quadrature point and 3k per element at N = 7
    assert bench._jvp_flops(_Case(7, 187_989, 38_250)) == 2 * (4 * 6300 + 3000) * 187_989
    assert abs(bench._jvp_flops(_Case(7, 187_989, 38_250)) - 1.06e10) < 0.01e10
    assert bench._jvp_flops(_Case(3, 10, 5)) is None


def test_tau_dd_instruction_model():
    import bench
    # per point at N = 7 (n = 13, t = 91): 15 instructions per double-float
    # multiply-add for M (3 t n), the second Gram matrix, B and tau (t n each)
    # and the four full products (n^3 each), 13 for the first Gram matrix (t n)
    per_point = 15 * (3 * 91 * 13 + 3 * 91 * 13 + 4 * 13 ** 3) + 13 * 91 * 13
    assert per_point == 253_669
    assert bench._tau_dd_instr(_Case(7, 10, 5)) == 4 * 10 * per_point
    # N = 1: one mode, n = t = 1
    assert bench._tau_dd_instr(_Case(1, 1, 4)) == 4 * (15 * (6 + 4) + 13)


def test_job_rate_counts_every_replica():
    import bench
    assert bench._job_rate(1, 100, 7, 31, 2.0) == 100 * 7 * 31 / 2.0
    assert bench._job_rate(4, 100, 7, 31, 2.0) == 4 * bench._job_rate(1, 100, 7, 31, 2.0)


def test_mode_error_is_the_space_time_l2_error():
    import numpy as np

    import bench
    # Parseval on the real signal u(t) = u_0 + 2 Re sum_n u_n e^{i n t}: the
    # mode-space error equals the time-sampled L2 error over one period
    rng = np.random.default_rng(3)
    ref = rng.standard_normal((6, 4, 5, 2))
    ref[:, :, 0, 1] = 0.0
    yN = ref[:, :, :3] + 0.01 * rng.standard_normal((6, 4, 3, 2))
    yN[:, :, 0, 1] = 0.0
    K = 64
    t = 2 * np.pi * np.arange(K) / K

    def samples(y):
        c = y[..., 0] + 1j * y[..., 1]
        n = np.arange(y.shape[2])
        s = np.real(c[..., :1]) + 2 * np.real(np.einsum("vfn,kn->vfk", c[..., 1:], np.exp(1j * np.outer(t, n[1:]))))
        return s[:, 0:3]

    err_t = np.sqrt(np.mean(np.sum((samples(ref) - np.pad(samples(yN), 0)) ** 2, axis=(0, 1))))
    norm_t = np.sqrt(np.mean(np.sum(samples(ref) ** 2, axis=(0, 1))))
    assert abs(bench.mode_error(yN, ref) - err_t / norm_t) < 1e-12
    assert bench.mode_error(ref, ref) == 0.0
