"""SSFM / ESSFM digital backpropagation with overlap-and-save (oracle, float64).

Follows Section II (Eqs. 1-3 and the step chaining after Eq. 2) and the
overlap-and-save description of Section III, step by step, with no fusion:

for each block of N vector samples (both polarizations), for each step s:
  (i)   X = DFT(x) per polarization                      (own radix-2 FFT)
  (ii)  Y_k = X_k H_s(f_k)                                (Eq. 1, inverted for DBP)
  (iii) y = IDFT(Y) per polarization
  (iv)  z_k = y_k exp(+j theta_k)                         (Eq. 2 or Eq. 3, inverted)
then keep the central N - O samples of each block.

Readings of the paper: backpropagation inverts the paper's forward operators,
i.e. H_s = exp(+j 2 pi^2 beta2 f^2 dz_s) and a +j nonlinear phase; the order inside a
step stays the paper's (linear, then nonlinear); the ESSFM filter indices k-i, k+i are
circular inside the block (the wrapped values land in the discarded overlap).
"""
from __future__ import annotations

import numpy as np

from . import dft
from .fiber import DBPConfig


def dispersion_tf(n: int, fs: float, beta2: float, dz: float, backward: bool = True) -> np.ndarray:
    """Eq. 1 transfer function exp(-j 2 pi^2 beta2 f_k^2 dz); its inverse when backward."""
    f = dft.fftfreq(n, fs)
    phase = 2.0 * np.pi ** 2 * beta2 * f ** 2 * dz
    return np.exp(1j * phase) if backward else np.exp(-1j * phase)


def linear_substep(x: np.ndarray, fs: float, beta2: float, dz: float, backward: bool = True) -> np.ndarray:
    """Operations (i)-(iii) of Section II on the last axis: FFT, times H, IFFT."""
    h = dispersion_tf(x.shape[-1], fs, beta2, dz, backward)
    return dft.ifft(dft.fft(x) * h)


def joint_intensity(y: np.ndarray) -> np.ndarray:
    """|y_k|^2 of a vector sample: sum over the two polarizations (axis -2)."""
    return np.sum(np.abs(y) ** 2, axis=-2)


def nl_substep_ssfm(y: np.ndarray, gamma_eff: float, backward: bool = True) -> np.ndarray:
    """Eq. 2: z_k = y_k exp(-j gamma dz_eff |y_k|^2), sign flipped when backward."""
    theta = gamma_eff * joint_intensity(y)
    sgn = 1.0 if backward else -1.0
    return y * np.exp(1j * sgn * theta)[..., None, :]


def essfm_phase(p: np.ndarray, gamma_eff: float, c: np.ndarray) -> np.ndarray:
    """Eq. 3 exponent (without the sign): gamma dz_eff (c_0 P_k + sum_i c_i (P_{k-i} + P_{k+i})),
    indices circular along the last axis."""
    theta = c[0] * p
    for i in range(1, len(c)):
        theta = theta + c[i] * (np.roll(p, i, axis=-1) + np.roll(p, -i, axis=-1))
    return gamma_eff * theta


def nl_substep_essfm(y: np.ndarray, gamma_eff: float, c: np.ndarray, backward: bool = True) -> np.ndarray:
    """Eq. 3: one common phase for both polarizations from the filtered joint intensity."""
    theta = essfm_phase(joint_intensity(y), gamma_eff, c)
    sgn = 1.0 if backward else -1.0
    return y * np.exp(1j * sgn * theta)[..., None, :]


def dbp_block(xb: np.ndarray, cfg: DBPConfig) -> np.ndarray:
    """All N_s steps on blocks xb [..., 2, N] (Section II step chaining)."""
    x = np.asarray(xb, dtype=np.complex128)
    for s in range(cfg.n_steps):
        y = linear_substep(x, cfg.fs, cfg.beta2, cfg.dz[s], backward=True)
        if cfg.essfm:
            x = nl_substep_essfm(y, cfg.gamma_eff[s], cfg.coeffs[s], backward=True)
        else:
            x = nl_substep_ssfm(y, cfg.gamma_eff[s] * cfg.coeffs[s][0], backward=True)
    return x


def block_layout(n: int, fft_size: int, overlap: int):
    """Overlap-and-save geometry (Section III): valid length V = N - O, number of
    blocks ceil(n / V), block b reads input window [b V - O/2, b V - O/2 + N)."""
    if overlap % 2 or overlap >= fft_size:
        raise ValueError("overlap must be even and smaller than the block length")
    v = fft_size - overlap
    nb = -(-n // v)
    starts = np.arange(nb) * v - overlap // 2
    return v, nb, starts


def gather_blocks(r: np.ndarray, cfg: DBPConfig, block_ids=None) -> np.ndarray:
    """Input windows [..., nb, 2, N]; outside [0, n) the waveform is periodic or zero."""
    n = r.shape[-1]
    v, nb, starts = block_layout(n, cfg.fft_size, cfg.overlap)
    ids = np.arange(nb) if block_ids is None else np.asarray(block_ids)
    idx = starts[ids][:, None] + np.arange(cfg.fft_size)[None, :]
    if cfg.boundary == "periodic":
        g = r[..., idx % n]                             # [..., 2, nb, N]
    else:
        inside = (idx >= 0) & (idx < n)
        g = np.where(inside, r[..., np.clip(idx, 0, n - 1)], 0.0)
    return np.moveaxis(g, -3, -2)                     # [..., nb, 2, N]


def dbp_blocks(r: np.ndarray, cfg: DBPConfig, block_ids) -> np.ndarray:
    """Valid outputs [..., len(ids), 2, N - O] of the listed blocks only."""
    xb = gather_blocks(np.asarray(r, dtype=np.complex128), cfg, block_ids)
    zb = dbp_block(xb, cfg)
    h = cfg.overlap // 2
    return zb[..., h:cfg.fft_size - h]


def dbp(r: np.ndarray, cfg: DBPConfig) -> np.ndarray:
    """Overlap-and-save DBP of waveforms r [..., 2, n]; returns [..., 2, n] complex128."""
    r = np.asarray(r, dtype=np.complex128)
    n = r.shape[-1]
    v, nb, _ = block_layout(n, cfg.fft_size, cfg.overlap)
    zc = dbp_blocks(r, cfg, np.arange(nb))             # [..., nb, 2, V]
    zc = np.moveaxis(zc, -3, -2)                       # [..., 2, nb, V]
    out = zc.reshape(zc.shape[:-2] + (nb * v,))
    return out[..., :n]


def dbp_per_step(r: np.ndarray, cfgs) -> np.ndarray:
    """Per-step-pass scheme: each step is a separate overlap-and-save pass over the whole
    waveform (one single-step config per step, in order from the receiver)."""
    x = np.asarray(r, dtype=np.complex128)
    for cfg in cfgs:
        x = dbp(x, cfg)
    return x
