"""Pins for oracle.spectral: the convolution matrix of eq. (phi-def)."""
import numpy as np

from oracle.spectral import conv_matrix, omega_diag, to_complex, to_storage


def _random_conj_sym(rng, N, batch=()):
    y = rng.standard_normal(batch + (N, 2))
    y[..., 0, 1] = 0.0
    return to_complex(y, N)


def _sampled_truncated_product(a, x, N, K):
    """Brute force: sample both signals at K points, multiply, take modes |m| < N."""
    def samples(c):
        t = np.arange(K) / K
        m = np.arange(-(N - 1), N)
        return (c[None, :] * np.exp(2j * np.pi * np.outer(t, m))).sum(axis=1)
    prod = samples(a) * samples(x)
    coef = np.fft.fft(prod) / K            # coef[k] = mode k (mod K)
    m = np.arange(-(N - 1), N)
    return coef[m % K]


def test_conv_matrix_equals_truncated_product_of_samples():
    rng = np.random.default_rng(0)
    for N in (1, 2, 3, 5, 7):
        a = _random_conj_sym(rng, N)
        x = _random_conj_sym(rng, N)
        ref = _sampled_truncated_product(a, x, N, K=4 * N)
        np.testing.assert_allclose(conv_matrix(a) @ x, ref, atol=1e-13, rtol=0)


def test_conv_matrix_aliases_with_too_few_samples():
    # with only 2N-1 samples the product aliases into the kept modes
    rng = np.random.default_rng(1)
    N = 4
    a = _random_conj_sym(rng, N)
    x = _random_conj_sym(rng, N)
    exact = conv_matrix(a) @ x
    assert np.abs(_sampled_truncated_product(a, x, N, K=2 * N - 1) - exact).max() > 1e-3
    np.testing.assert_allclose(_sampled_truncated_product(a, x, N, K=3 * N - 2), exact, atol=1e-13)


def test_conv_matrix_hermitian_toeplitz_corners_zero():
    rng = np.random.default_rng(2)
    N = 5
    a = _random_conj_sym(rng, N)
    A = conv_matrix(a)
    np.testing.assert_allclose(A, A.conj().T, atol=0)
    for k in range(1, 2 * N - 1):
        d = np.diagonal(A, offset=-k)
        if k < N:
            np.testing.assert_allclose(d, a[N - 1 + k])
        else:
            assert np.all(d == 0)


def test_storage_round_trip_and_conjugate_symmetry():
    rng = np.random.default_rng(3)
    N = 4
    y = rng.standard_normal((6, N, 2))
    y[:, 0, 1] = 0.0
    x = to_complex(y, N)
    np.testing.assert_allclose(x[:, : N - 1], np.conj(x[:, N:][:, ::-1]))
    np.testing.assert_allclose(to_storage(x, N), y)


def test_omega_skew_hermitian():
    w = omega_diag(4, 0.7)
    Om = np.diag(w)
    np.testing.assert_allclose(Om.conj().T, -Om)
    rng = np.random.default_rng(4)
    x = _random_conj_sym(rng, 4)
    assert abs((x.conj() @ Om @ x).real) < 1e-14   # (w, Omega w) = 0, Lemma 1
