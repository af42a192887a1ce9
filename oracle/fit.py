"""ESSFM coefficient optimisation by minimum MSE (oracle, float64).

Section IV: the coefficients are chosen to minimise the mean square error between
the ESSFM output and a target (the output of a many-step SSFM, or -- footnote of
Section IV -- the transmitted signal) over a training part of the waveform.  For a
single step (N_s = 1) the linear sub-step output y does not depend on c, and the
output z = y exp(j theta), theta = gamma_eff sum_i c_i S_i (S_0 = P_k,
S_i = P_{k-i} + P_{k+i}) is fitted by Gauss-Newton on the complex residual
t - z: dz/dc_i = j gamma_eff S_i z.  The start point is the SSFM (c = [1, 0, ...]).
"""
from __future__ import annotations

import numpy as np

from . import dbp as odbp
from .fiber import DBPConfig


def _regressors(y: np.ndarray, gamma_eff: float, n_taps: int) -> np.ndarray:
    p = odbp.joint_intensity(y)                       # [nb, N]
    s = [p]
    for i in range(1, n_taps + 1):
        s.append(np.roll(p, i, axis=-1) + np.roll(p, -i, axis=-1))
    return gamma_eff * np.stack(s, axis=-1)           # [nb, N, Nc+1]


def fit_single_step(r: np.ndarray, target: np.ndarray, cfg: DBPConfig, n_train=None,
                    n_iter: int = 20, tol: float = 1e-13) -> np.ndarray:
    """Fit c_0..c_Nc of a 1-step ESSFM on waveform r [2, n] against target [2, n] over
    the first n_train output samples.  Returns float64 [Nc+1]."""
    if cfg.n_steps != 1:
        raise ValueError("closed-form Gauss-Newton fit is for a single step")
    n = r.shape[-1]
    n_train = n if n_train is None else n_train
    v, nb, _ = odbp.block_layout(n, cfg.fft_size, cfg.overlap)
    xb = odbp.gather_blocks(np.asarray(r, dtype=np.complex128), cfg)       # [nb, 2, N]
    y = odbp.linear_substep(xb, cfg.fs, cfg.beta2, cfg.dz[0], backward=True)
    h = cfg.overlap // 2
    reg = _regressors(y, cfg.gamma_eff[0], cfg.n_taps)[:, h:h + v, :]      # [nb, V, K]
    yv = y[..., h:h + v]                                                   # [nb, 2, V]
    # target laid out like the valid outputs of each block
    pos = (np.arange(nb)[:, None] * v + np.arange(v)[None, :])             # [nb, V]
    keep = pos < min(n, n_train)
    t = np.asarray(target, dtype=np.complex128)[:, np.clip(pos, 0, n - 1)]  # [2, nb, V]
    t = np.moveaxis(t, 0, 1)                                                 # [nb, 2, V]
    regk = reg[keep]                                                         # [m, K]
    yk = np.moveaxis(yv, 1, 2)[keep]                                         # [m, 2]
    tk = np.moveaxis(t, 1, 2)[keep]                                          # [m, 2]
    c = np.zeros(cfg.n_taps + 1)
    c[0] = 1.0
    for _ in range(n_iter):
        theta = regk @ c                                                     # [m]
        z = yk * np.exp(1j * theta)[:, None]
        e = (tk - z).reshape(-1)
        jac = (1j * z[:, :, None] * regk[:, None, :]).reshape(-1, c.size)    # [2m, K]
        a = np.concatenate([jac.real, jac.imag], axis=0)
        b = np.concatenate([e.real, e.imag], axis=0)
        delta, *_ = np.linalg.lstsq(a, b, rcond=None)
        c = c + delta
        if np.max(np.abs(delta)) < tol * max(1.0, np.max(np.abs(c))):
            break
    return c
