"""Operation-count model of Section III (context numbers and the autotuner's prior).

Per step and per received sample, with block length N and M discarded samples:
  ESSFM:  N (8 log2 N + 21 + N_c) / (N - M) real multiplications,
          N (8 log2 N + 11 + 2 N_c) / (N - M) real additions;
  SSFM:   the same with N_c = 0;
  FFE:    N (8 log2 N + 8) / (N - M) multiplications, N (8 log2 N + 4) / (N - M) additions.
The paper counts a radix-2 FFT (8 N log2 N real multiplications and additions for the
four N-point FFTs of a step) and a table-lookup exponential.
"""
from __future__ import annotations

import math


def mults_per_sample(n: float, m: float, n_taps: int = 0, ffe: bool = False) -> float:
    """Real multiplications per step per received sample (Section III)."""
    if n <= m:
        raise ValueError("block length must exceed the overlap")
    core = 8.0 * math.log2(n)
    extra = 8.0 if ffe else 21.0 + n_taps
    return n * (core + extra) / (n - m)


def adds_per_sample(n: float, m: float, n_taps: int = 0, ffe: bool = False) -> float:
    """Real additions per step per received sample (Section III)."""
    if n <= m:
        raise ValueError("block length must exceed the overlap")
    core = 8.0 * math.log2(n)
    extra = 4.0 if ffe else 11.0 + 2 * n_taps
    return n * (core + extra) / (n - m)


def total_mults(n: float, m: float, n_steps: int, n_taps: int = 0) -> float:
    """All steps: N_s times the per-step count (Section III, Fig. 1/2 discussion)."""
    return n_steps * mults_per_sample(n, m, n_taps)


def memory_samples(beta2_s2_per_m: float, length_m: float, bandwidth_hz: float) -> float:
    """Section III: M ~= 2 pi |beta2| L B^2."""
    return 2.0 * math.pi * abs(beta2_s2_per_m) * length_m * bandwidth_hz ** 2
