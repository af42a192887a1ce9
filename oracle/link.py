"""Forward Manakov channel simulator with ideal EDFAs and ASE (oracle, float64).

Test-vector generator for the backpropagation checks; it is the forward counterpart
of Section II: per small sub-step h of each span, a nonlinear phase rotation
exp(-j gamma m |u|^2 h_eff) common to both polarizations (Manakov, Section II, with
m the 8/9 factor) and a linear step exp(-j beta2 w^2 h / 2) with field attenuation
exp(-alpha h / 2) (the paper's sign convention of Eqs. 1-2).  Symmetric (Strang)
splitting: half linear, nonlinear at the midpoint, half linear.  Each span ends in an
ideal EDFA of gain G = exp(alpha L_span) followed by circular complex Gaussian ASE of
variance n_sp h nu (G - 1) f_s per sample per polarization, n_sp = F G / (2 (G - 1))
(F the noise figure).  The full waveform is treated as periodic.  numpy's FFT serves
as the DFT primitive here (library routine); the DBP oracle uses its own FFT.
"""
from __future__ import annotations

import math

import numpy as np

from .fiber import C_LIGHT, H_PLANCK, alpha_per_m, beta2_from_D


def _lin(u, fs, beta2, alpha, h, inverse=False):
    n = u.shape[-1]
    w = 2.0 * np.pi * np.fft.fftfreq(n, 1.0 / fs)
    if not inverse:
        tf = np.exp(-1j * beta2 * w ** 2 * h / 2.0) * math.exp(-alpha * h / 2.0)
    else:
        tf = np.exp(+1j * beta2 * w ** 2 * h / 2.0) * math.exp(+alpha * h / 2.0)
    return np.fft.ifft(np.fft.fft(u, axis=-1) * tf, axis=-1)


def _nl(u, g_heff, inverse=False):
    p = np.sum(np.abs(u) ** 2, axis=-2, keepdims=True)
    sgn = 1.0 if inverse else -1.0
    return u * np.exp(1j * sgn * g_heff * p)


def _mid_heff(alpha, h):
    """Integral over the sub-step of the power relative to its midpoint value."""
    if alpha == 0.0:
        return h
    return math.exp(alpha * h / 2.0) * (1.0 - math.exp(-alpha * h)) / alpha


def ase_variance(link: dict, fs: float) -> float:
    """ASE power per sample per polarization added by one EDFA."""
    alpha = alpha_per_m(link["alpha_db_per_km"])
    g = math.exp(alpha * link["span_len_m"])
    f_nf = 10.0 ** (link.get("nf_db", 5.0) / 10.0)
    nsp = f_nf * g / (2.0 * (g - 1.0))
    nu = C_LIGHT / link["lambda_m"]
    return nsp * H_PLANCK * nu * (g - 1.0) * fs


def forward(tx: np.ndarray, link: dict, fs: float, steps_per_span: int = 1000,
            ase_seed=None, gamma_scale: float = 1.0) -> np.ndarray:
    """Propagate tx [..., 2, n] through ``link``; ASE added only if ase_seed is not None."""
    u = np.asarray(tx, dtype=np.complex128).copy()
    alpha = alpha_per_m(link["alpha_db_per_km"])
    beta2 = beta2_from_D(link["D_ps_per_nm_km"], link["lambda_m"])
    gamma = link["gamma_per_W_km"] * 1e-3 * link.get("manakov_factor", 1.0) * gamma_scale
    h = link["span_len_m"] / steps_per_span
    g_heff = gamma * _mid_heff(alpha, h)
    gain = math.exp(alpha * link["span_len_m"])
    rng = None if ase_seed is None else np.random.default_rng(np.random.PCG64(ase_seed))
    var = ase_variance(link, fs)
    for _ in range(link["n_spans"]):
        for _ in range(steps_per_span):
            u = _lin(u, fs, beta2, alpha, h / 2.0)
            u = _nl(u, g_heff)
            u = _lin(u, fs, beta2, alpha, h / 2.0)
        u = u * math.sqrt(gain)
        if rng is not None:
            s = math.sqrt(var / 2.0)
            u = u + s * (rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape))
    return u


def inverse(rx: np.ndarray, link: dict, fs: float, steps_per_span: int = 1000,
            gamma_scale: float = 1.0) -> np.ndarray:
    """Exact inverse of ``forward`` without ASE: every sub-operator undone in reverse."""
    u = np.asarray(rx, dtype=np.complex128).copy()
    alpha = alpha_per_m(link["alpha_db_per_km"])
    beta2 = beta2_from_D(link["D_ps_per_nm_km"], link["lambda_m"])
    gamma = link["gamma_per_W_km"] * 1e-3 * link.get("manakov_factor", 1.0) * gamma_scale
    h = link["span_len_m"] / steps_per_span
    g_heff = gamma * _mid_heff(alpha, h)
    gain = math.exp(alpha * link["span_len_m"])
    for _ in range(link["n_spans"]):
        u = u / math.sqrt(gain)
        for _ in range(steps_per_span):
            u = _lin(u, fs, beta2, alpha, h / 2.0, inverse=True)
            u = _nl(u, g_heff, inverse=True)
            u = _lin(u, fs, beta2, alpha, h / 2.0, inverse=True)
    return u
