"""Mode vectors and the mode matrices of section 2.1 (eq. phi-def).

A field with N independent modes is stored as 2N-1 complex coefficients
x_m, m = -N+1..N-1, at index m + N - 1.  Real-valued time signals give
x_{-m} = conj(x_m) (section 2.1, below eq. phiDef).

Pinned by: tests/test_oracle_spectral.py (convolution matrix equals the
truncated product of the sampled time signals, computed with a library FFT;
Hermitian Toeplitz structure; storage round trip).
"""
from __future__ import annotations

import numpy as np


def n_modes(N: int) -> int:
    return 2 * N - 1


def to_complex(y: np.ndarray, N: int) -> np.ndarray:
    """Storage [..., N, 2] (re, im of modes 0..N-1) -> full complex [..., 2N-1].

    The imaginary part stored for mode 0 is ignored (mode 0 of a real signal
    is real; section 2.5.1 keeps that slot only for layout).
    """
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros(y.shape[:-2] + (2 * N - 1,), dtype=np.complex128)
    pos = y[..., :, 0] + 1j * y[..., :, 1]
    pos[..., 0] = y[..., 0, 0]
    out[..., N - 1:] = pos
    out[..., : N - 1] = np.conj(pos[..., 1:][..., ::-1])
    return out


def to_storage(x: np.ndarray, N: int, keep_im0: bool = False) -> np.ndarray:
    """Full complex [..., 2N-1] -> storage [..., N, 2]; Im of mode 0 zeroed unless asked."""
    pos = x[..., N - 1:]
    out = np.stack([pos.real, pos.imag], axis=-1)
    if not keep_im0:
        out[..., 0, 1] = 0.0
    return out


def conv_matrix(a: np.ndarray) -> np.ndarray:
    """A_{mn} = a_{m-n} for |m-n| < N, zero otherwise (eq. phi-def).

    ``a`` is [..., 2N-1]; the result is [..., 2N-1, 2N-1].
    """
    nm = a.shape[-1]
    N = (nm + 1) // 2
    m = np.arange(-(N - 1), N)
    k = m[:, None] - m[None, :]                   # m - n
    valid = np.abs(k) < N
    idx = np.where(valid, k + N - 1, 0)
    A = a[..., idx]
    return np.where(valid, A, 0.0)


def omega_diag(N: int, omega: float) -> np.ndarray:
    """Diagonal of Omega: Omega_mm = i m omega (eq. phi-def)."""
    m = np.arange(-(N - 1), N)
    return 1j * m * omega
