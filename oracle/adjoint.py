"""Reverse-mode gradient (vector-Jacobian product) of the overlap-save DBP (oracle, float64).

For a real loss L of the DBP output and g_out = dL/dRe(out) + j dL/dIm(out), returns
the gradients with respect to the input waveform, the ESSFM coefficients c_{s,i}, the
per-step nonlinear strengths gamma_eff_s and the per-step lengths dz_s (which enter
only through H_s; gamma_eff_s is an independent parameter).  Derived by hand from the
forward operators of Section II (Eqs. 1-3) and the overlap-and-save of Section III:

* nonlinear step z = y exp(j theta): s_k = dL/dtheta_k = -sum_p Im(conj(g_z) z);
  dL/dc_i = gamma sum_k s_k S_{k,i}; dL/dgamma = sum_k s_k theta_k / gamma;
  dL/dP = the same symmetric filter applied to s; g_y = g_z exp(-j theta) + 2 (dL/dP) y.
* linear step y = IDFT(H DFT(x)) is unitary: g_x = IDFT(conj(H) DFT(g_y));
  dL/ddz = sum_k Re(conj(G_k) j phi'_k Y_k) / N with G = DFT(g_y), Y = H DFT(x),
  phi'_k = 2 pi^2 beta2 f_k^2.
* overlap-and-save transposes to overlap-add of the block input gradients.
"""
from __future__ import annotations

import numpy as np

from . import dbp as odbp
from . import dft
from .fiber import DBPConfig


def dbp_vjp(r: np.ndarray, cfg: DBPConfig, g_out: np.ndarray):
    """Returns (g_in [2, n], g_coeffs [N_s, N_c+1], g_gamma_eff [N_s], g_dz [N_s])."""
    r = np.asarray(r, dtype=np.complex128)
    g_out = np.asarray(g_out, dtype=np.complex128)
    n = r.shape[-1]
    nn, o = cfg.fft_size, cfg.overlap
    v, nb, starts = odbp.block_layout(n, nn, o)
    h = o // 2
    x = odbp.gather_blocks(r, cfg)                     # [nb, 2, N]
    f = dft.fftfreq(nn, cfg.fs)
    dphi = 2.0 * np.pi ** 2 * cfg.beta2 * f ** 2       # d(phase)/d(dz)
    n_c = cfg.n_taps if cfg.essfm else 0

    # forward sweep, keeping each step's block input (checkpoints)
    ckpt = []
    for s in range(cfg.n_steps):
        ckpt.append(x)
        y = odbp.linear_substep(x, cfg.fs, cfg.beta2, cfg.dz[s], backward=True)
        c = cfg.coeffs[s][: n_c + 1]
        theta = odbp.essfm_phase(odbp.joint_intensity(y), cfg.gamma_eff[s], c)
        x = y * np.exp(1j * theta)[:, None, :]

    # output gradient placed in each block's valid (central) region
    pos = np.arange(nb)[:, None] * v + np.arange(v)[None, :]
    inside = pos < n
    gz = np.zeros((nb, 2, nn), dtype=np.complex128)
    gsel = g_out[:, np.clip(pos, 0, n - 1)]            # [2, nb, V]
    gz[:, :, h:h + v] = np.where(inside[None], gsel, 0.0).transpose(1, 0, 2)

    g_c = np.zeros_like(cfg.coeffs)
    g_gamma = np.zeros(cfg.n_steps)
    g_dz = np.zeros(cfg.n_steps)
    for s in reversed(range(cfg.n_steps)):
        xs = ckpt[s]
        hs = odbp.dispersion_tf(nn, cfg.fs, cfg.beta2, cfg.dz[s], backward=True)
        xf = dft.fft(xs)
        yf = xf * hs
        y = dft.ifft(yf)
        p = odbp.joint_intensity(y)
        c = cfg.coeffs[s][: n_c + 1]
        g = cfg.gamma_eff[s]
        theta = odbp.essfm_phase(p, g, c)
        z = y * np.exp(1j * theta)[:, None, :]
        sk = -np.sum(np.imag(np.conj(gz) * z), axis=1)             # [nb, N]
        g_c[s, 0] += g * np.sum(sk * p)
        for i in range(1, n_c + 1):
            g_c[s, i] += g * np.sum(sk * (np.roll(p, i, axis=-1) + np.roll(p, -i, axis=-1)))
        g_gamma[s] += np.sum(sk * theta) / g if g != 0.0 else np.sum(
            sk * odbp.essfm_phase(p, 1.0, c))
        dldp = odbp.essfm_phase(sk, g, c)
        gy = gz * np.exp(-1j * theta)[:, None, :] + 2.0 * dldp[:, None, :] * y
        gf = dft.fft(gy)
        g_dz[s] += np.sum(np.real(np.conj(gf) * 1j * dphi * yf)) / nn
        gz = dft.ifft(np.conj(hs) * gf)

    # overlap-add of block input gradients
    g_in = np.zeros((2, n), dtype=np.complex128)
    idx = starts[:, None] + np.arange(nn)[None, :]
    for b in range(nb):
        ib = idx[b]
        if cfg.boundary == "periodic":
            np.add.at(g_in, (slice(None), ib % n), gz[b])
        else:
            ok = (ib >= 0) & (ib < n)
            np.add.at(g_in, (slice(None), ib[ok]), gz[b][:, ok])
    return g_in, g_c, g_gamma, g_dz
