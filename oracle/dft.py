"""Naive DFT and an own radix-2 FFT, float64 (oracle; test infrastructure only).

Convention (as numpy): X_k = sum_n x_n exp(-j 2 pi n k / N),
x_n = (1/N) sum_k X_k exp(+j 2 pi n k / N).  The paper counts operations for the
classical Cooley-Tukey radix-2 FFT (Section III footnote); ``fft`` below is that
algorithm (decimation in time, bit-reversed input order), vectorised only over
leading axes.
"""
from __future__ import annotations

import numpy as np


def naive_dft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Definition of the DFT along the last axis (O(N^2)).  The angle uses the exact
    integer (n k mod N) so the matrix entries are correctly rounded."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    k = np.arange(n)
    nk = np.outer(k, k) % n
    sign = 1.0 if inverse else -1.0
    w = np.exp(sign * 2j * np.pi * nk / n)
    y = x @ w.T
    return y / n if inverse else y


def _bit_reverse(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft(x: np.ndarray) -> np.ndarray:
    """Radix-2 decimation-in-time Cooley-Tukey FFT along the last axis."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n & (n - 1):
        raise ValueError("fft length must be a power of two")
    a = x[..., _bit_reverse(n)]
    lead = a.shape[:-1]
    m = 1
    while m < n:
        # groups of 2m: first m entries are the even-index sub-DFT, next m the odd one
        a = a.reshape(lead + (n // (2 * m), 2, m))
        w = np.exp(-1j * np.pi * np.arange(m) / m)      # W_{2m}^k
        even = a[..., 0, :]
        odd = a[..., 1, :] * w
        a = np.concatenate([even + odd, even - odd], axis=-1)
        m *= 2
    return a.reshape(lead + (n,))


def ifft(x: np.ndarray) -> np.ndarray:
    """Inverse via conjugation: IDFT(X) = conj(DFT(conj X)) / N."""
    x = np.asarray(x, dtype=np.complex128)
    return np.conj(fft(np.conj(x))) / x.shape[-1]


def fftfreq(n: int, fs: float) -> np.ndarray:
    """Frequency of bin k: k fs/N for k < N/2, (k - N) fs/N otherwise."""
    k = np.arange(n)
    return np.where(k < n // 2, k, k - n) * (fs / n)
