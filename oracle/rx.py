"""Minimal synthetic receiver (oracle, float64): matched filter, symbol sampling,
data-aided gain, Gray QPSK decisions, BER and Q-factor.

Stands in for the offline chain of Section IV (resampling, butterfly equaliser,
asynchronous detection, decisions), which corrects impairments the synthetic link
does not have (PMD, laser phase noise, frequency offset).  Readings:
one least-squares complex gain per polarization against the transmitted symbols;
Q_dB = 10 log10(SNR_eff) with SNR_eff = E|s|^2 / E|s_hat - s|^2 (for Gray QPSK in
Gaussian noise BER = erfc(Q / sqrt 2) / 2 with Q^2 = SNR); decisions take the sign
bit (x >= 0 -> bit 0).
"""
from __future__ import annotations

import math

import numpy as np


def raised_cosine_sqrt(n: int, sps: int, rolloff: float) -> np.ndarray:
    """Square root of the raised-cosine spectrum on the FFT grid of n samples."""
    f = np.abs(np.fft.fftfreq(n, d=1.0 / sps))          # units of the symbol rate
    lo, hi = 0.5 * (1.0 - rolloff), 0.5 * (1.0 + rolloff)
    rc = np.where(f <= lo, 1.0, 0.0)
    band = (f > lo) & (f < hi)
    rc = np.where(band, 0.5 * (1.0 - np.sin(np.pi * (f - 0.5) / rolloff)), rc)
    return np.sqrt(np.clip(rc, 0.0, None))


def matched_filter(x: np.ndarray, sps: int = 2, rolloff: float = 0.1) -> np.ndarray:
    h = raised_cosine_sqrt(x.shape[-1], sps, rolloff)
    return np.fft.ifft(np.fft.fft(x, axis=-1) * h, axis=-1)


def symbols_out(x: np.ndarray, sps: int = 2, rolloff: float = 0.1) -> np.ndarray:
    """Matched-filtered samples at the symbol centres, [..., 2, n/sps]."""
    return matched_filter(np.asarray(x, dtype=np.complex128), sps, rolloff)[..., ::sps]


def equalise(r: np.ndarray, s: np.ndarray) -> np.ndarray:
    """One LS complex gain per polarization: s_hat = r / g, g = <s, r> / <s, s>."""
    g = np.sum(np.conj(s) * r, axis=-1, keepdims=True) / np.sum(np.abs(s) ** 2, axis=-1, keepdims=True)
    return r / g


def decide(s_hat: np.ndarray) -> np.ndarray:
    bits = np.empty(s_hat.shape + (2,), dtype=np.uint8)
    bits[..., 0] = (s_hat.real < 0).astype(np.uint8)
    bits[..., 1] = (s_hat.imag < 0).astype(np.uint8)
    return bits


def evaluate(x: np.ndarray, tx_symbols: np.ndarray, tx_bits: np.ndarray,
             sps: int = 2, rolloff: float = 0.1, skip: int = 0) -> dict:
    """BER, SNR_eff and Q (dB) of a received waveform x [2, n] against the transmitted
    symbols/bits; the first ``skip`` symbols are excluded (training part)."""
    r = symbols_out(x, sps, rolloff)[..., skip:]
    s = tx_symbols[..., skip:]
    s_hat = equalise(r, s)
    err = np.mean(np.abs(s_hat - s) ** 2)
    snr = np.mean(np.abs(s) ** 2) / err
    bits = decide(s_hat)
    n_err = int(np.sum(bits != tx_bits[..., skip:, :]))
    n_bits = bits.size
    ber = n_err / n_bits
    return dict(ber=ber, bit_errors=n_err, bits=n_bits, snr_eff=snr,
                q_db=10.0 * math.log10(snr), decisions=bits, s_hat=s_hat)
