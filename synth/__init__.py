"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *generates inputs*: polarization-multiplexed QPSK symbols,
root-raised-cosine pulse shaping at 2 samples/symbol, launch-power scaling,
additive white Gaussian noise and the link/signal parameter sets of the
workloads.  It holds none of the backpropagation arithmetic (no dispersion
operator, no nonlinear step, no step table, no overlap rule) and imports
neither the oracle nor the CUDA package.

The experiment of Section IV (112 Gb/s PM-QPSK, 28 GBaud, 3200 km of SMF in
80 km spans) is replaced by these seeded stand-ins; the lab data of Fig. 4 is
not available.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 150700921

# Physical parameters of the synthetic link (Section IV experiment stand-in):
# standard single-mode fibre, 80 km spans, ideal EDFAs with 5 dB noise figure.
SMF = dict(
    span_len_m=80e3,
    alpha_db_per_km=0.2,
    D_ps_per_nm_km=17.0,
    lambda_m=1550e-9,
    gamma_per_W_km=1.3,
    manakov_factor=8.0 / 9.0,
    nf_db=5.0,
)

SYMBOL_RATE = 28e9          # 28 GBaud per polarization (Section IV)
SPS = 2                     # samples per symbol
SAMPLE_RATE = SYMBOL_RATE * SPS
ROLLOFF = 0.1


def link(n_spans: int, **over) -> dict:
    """Link parameter set with ``n_spans`` x 80 km spans of SMF."""
    d = dict(SMF)
    d["n_spans"] = int(n_spans)
    d.update(over)
    return d


# The workloads: (a) 2^14 symbols over 10 spans, (b) 2^18 symbols over 40 spans.
WORKLOADS = {
    "cfg1_800km": dict(n_symbols=2 ** 14, n_spans=10, launch_dbm=2.0, fft_size=1024,
                       essfm=dict(n_steps=1, n_taps=8), ssfm=dict(n_steps=20, n_taps=0)),
    "cfg2_3200km": dict(n_symbols=2 ** 18, n_spans=40, launch_dbm=2.0, fft_size=4096,
                        essfm=dict(n_steps=1, n_taps=32), ssfm=dict(n_steps=20, n_taps=0)),
}


def dbm_to_w(p_dbm: float) -> float:
    return 1e-3 * 10.0 ** (p_dbm / 10.0)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def qpsk_bits(n_symbols: int, seed: int, n_pol: int = 2) -> np.ndarray:
    """Uniform random bits, shape [n_pol, n_symbols, 2] (uint8)."""
    return rng(seed).integers(0, 2, size=(n_pol, n_symbols, 2), dtype=np.uint8)


def qpsk_map(bits: np.ndarray) -> np.ndarray:
    """Gray-mapped unit-energy QPSK: bit 0 -> +, bit 1 -> - on each quadrature."""
    b = bits.astype(np.float64)
    return ((1.0 - 2.0 * b[..., 0]) + 1j * (1.0 - 2.0 * b[..., 1])) / np.sqrt(2.0)


def rrc_response(n: int, sps: int = SPS, rolloff: float = ROLLOFF) -> np.ndarray:
    """Frequency response (length n, FFT bin order) of a unit-gain root-raised-cosine
    filter for symbol period ``sps`` samples.  Used by the transmitter only."""
    f = np.fft.fftfreq(n) * sps            # frequency in units of the symbol rate
    af = np.abs(f)
    f1 = (1.0 - rolloff) / 2.0
    f2 = (1.0 + rolloff) / 2.0
    h = np.zeros(n)
    h[af <= f1] = 1.0
    mid = (af > f1) & (af < f2)
    h[mid] = np.sqrt(0.5 * (1.0 + np.cos(np.pi / rolloff * (af[mid] - f1))))
    return h


def pm_qpsk_waveform(n_symbols: int, seed: int, launch_dbm: float = 0.0,
                     sps: int = SPS, rolloff: float = ROLLOFF):
    """Seeded dual-polarization QPSK waveform.

    Returns ``(x, symbols, bits)``: ``x`` complex128 [2, n_symbols*sps] with mean
    power per polarization equal to the launch power (W); ``symbols`` [2, n_symbols];
    ``bits`` [2, n_symbols, 2].  Pulse shaping is circular (the waveform is periodic),
    matching a periodic channel simulation.
    """
    bits = qpsk_bits(n_symbols, seed)
    sym = qpsk_map(bits)
    n = n_symbols * sps
    up = np.zeros((2, n), dtype=np.complex128)
    up[:, ::sps] = sym
    x = np.fft.ifft(np.fft.fft(up, axis=-1) * rrc_response(n, sps, rolloff), axis=-1)
    p = dbm_to_w(launch_dbm)
    x *= np.sqrt(p / np.mean(np.abs(x) ** 2, axis=-1, keepdims=True))
    return x, sym, bits


def awgn(shape, var_per_sample: float, seed: int) -> np.ndarray:
    """Circular complex Gaussian noise with E|n|^2 = var_per_sample."""
    g = rng(seed)
    s = np.sqrt(var_per_sample / 2.0)
    return s * (g.standard_normal(shape) + 1j * g.standard_normal(shape))


def random_field(n_waveforms: int, n_samples: int, power_w: float, seed: int) -> np.ndarray:
    """Generic seeded Gaussian field [n_waveforms, 2, n_samples] (complex128) with
    mean power ``power_w`` per polarization: the amplitude statistics of a
    dispersed long-haul signal, used where only shape and scale matter."""
    return awgn((n_waveforms, 2, n_samples), power_w, seed)


def received_like(n_waveforms: int, n_symbols: int, launch_dbm: float, seed: int,
                  snr_db: float = 22.0, distinct: int = 8) -> np.ndarray:
    """Benchmark input: ``n_waveforms`` PM-QPSK waveforms [B, 2, 2*n_symbols]
    (complex64) at the launch power plus white noise at ``snr_db`` in-band SNR.
    ``distinct`` different seeds are generated and repeated across the batch."""
    n = n_symbols * SPS
    out = np.empty((n_waveforms, 2, n), dtype=np.complex64)
    p = dbm_to_w(launch_dbm)
    noise_var = p / 10.0 ** (snr_db / 10.0) * SPS      # in-band SNR -> per-sample variance
    cache = []
    for i in range(min(distinct, n_waveforms)):
        x, _, _ = pm_qpsk_waveform(n_symbols, seed + i, launch_dbm)
        x = x + awgn(x.shape, noise_var, seed + 1000 + i)
        cache.append(x.astype(np.complex64))
    for b in range(n_waveforms):
        out[b] = cache[b % len(cache)]
    return out


def batch_jobs(n_jobs: int, seed: int, min_log2_symbols: int = 12, max_log2_symbols: int = 18):
    """Seeded uneven job list for batched backpropagation: symbol counts log-uniform in
    [2^min, 2^max], links of 10/20/30/40 spans (800-3200 km), launch powers uniform in
    0-4 dBm, and a mix of multi-step SSFM (5-20 steps) and 1-2 step ESSFM (8-32 taps)."""
    g = rng(seed)
    jobs = []
    for j in range(n_jobs):
        log2s = g.uniform(min_log2_symbols, max_log2_symbols)
        n_sym = int(round(2.0 ** log2s))
        spans = int(g.choice([10, 20, 30, 40]))
        dbm = float(g.uniform(0.0, 4.0))
        if g.random() < 0.5:
            method, ns, nc = "ssfm", int(g.integers(5, 21)), 0
        else:
            method, ns, nc = "essfm", int(g.integers(1, 3)), int(g.choice([8, 16, 24, 32]))
        jobs.append(dict(n_symbols=n_sym, n_spans=spans, launch_dbm=dbm, method=method, n_steps=ns, n_taps=nc,
                         seed=seed + 10 * j))
    return jobs
