"""Fitting the ESSFM coefficients on the GPU (Section IV and its footnote).

Section IV fits the coefficients by minimum MSE against a many-step SSFM output; its
footnote suggests the MSE between the equalised output symbols and the transmitted
symbols instead.  ``fit_adam`` does the latter with gradients from libdbp's adjoint:
loss = mean over symbols and polarizations of |s_hat - s|^2, where s_hat are the
matched-filtered (root-raised-cosine) output samples at the symbol centres divided
by one least-squares complex gain per polarization (replacing the butterfly equaliser
and carrier recovery of the paper's receiver, which correct impairments a synthetic
link does not have).  The matched filter and gain are torch operations on the DBP
output; backpropagation itself runs in libdbp (forward kernel and adjoint kernel).
"""
from __future__ import annotations

import math

import numpy as np


def rrc_matched_response(n: int, sps: int = 2, rolloff: float = 0.1, device="cuda"):
    """Root-raised-cosine frequency response on the FFT grid of n samples."""
    import torch
    f = torch.fft.fftfreq(n, d=1.0 / sps, device=device).abs().double()
    lo, hi = 0.5 * (1 - rolloff), 0.5 * (1 + rolloff)
    h = torch.where(f <= lo, torch.ones_like(f), torch.zeros_like(f))
    band = (f > lo) & (f < hi)
    h = torch.where(band, torch.sqrt(0.5 * (1 - torch.sin(math.pi * (f - 0.5) / rolloff))), h)
    return h.float()


def symbol_mse(out, symbols, h_mf, sps: int = 2):
    """MSE of the gain-corrected matched-filter symbols against the transmitted ones."""
    import torch
    r = torch.fft.ifft(torch.fft.fft(out, dim=-1) * h_mf, dim=-1)[..., ::sps]
    g = (torch.conj(symbols) * r).sum(-1, keepdim=True) / (symbols.abs() ** 2).sum(-1, keepdim=True)
    return ((r / g - symbols).abs() ** 2).mean()


def fit_adam(plan, x, symbols, coeffs0=None, n_iter: int = 200, lr: float = 2e-3, sps: int = 2):
    """Adam on the ESSFM coefficients of ``plan`` for waveforms x [B, 2, n] (CUDA
    complex64) and transmitted symbols [B, 2, n/sps].  Returns (coeffs, losses)."""
    import torch
    from .dbp import DBP
    module = DBP(plan, coeffs0)
    opt = torch.optim.Adam(module.parameters(), lr=lr)
    h_mf = rrc_matched_response(x.shape[-1], sps, device=x.device)
    losses = []
    for _ in range(n_iter):
        opt.zero_grad()
        loss = symbol_mse(module(x), symbols, h_mf, sps)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    return module.coeffs.detach().cpu().numpy().astype(np.float32), losses



def fit_gauss_newton(link: dict, fs: float, x, target, n_taps: int, fft_size: int, n_train=None,
                     max_iter: int = 20, overlap: int = 0, boundary: str = "periodic", coeffs0=None,
                     common_phase: bool = False):
    """Section IV fit of a single-step ESSFM with N_c = ``n_taps`` and block length
    ``fft_size`` to ``target`` (minimum MSE, Gauss-Newton, on the GPU through
    dbp_fit_coeffs) from ``coeffs0`` (default the SSFM, c = 1, 0, ..., 0; c = 0 is the
    linear-only compensation), optionally with a common phase fitted alongside
    (``common_phase``).  x, target: CUDA complex64 [n_waveforms, 2, n] or [2, n].
    Returns ``(coeffs float64 [n_taps + 1], losses)`` (``(coeffs, losses, phase)`` with
    ``common_phase``)."""
    from .dbp import Plan
    xs = x if x.dim() == 3 else x.unsqueeze(0)
    ts = target if target.dim() == 3 else target.unsqueeze(0)
    with Plan(link, fs, xs.shape[-1], n_waveforms=xs.shape[0], method="essfm", n_steps=1, n_taps=n_taps,
              fft_size=fft_size, overlap=overlap, boundary=boundary) as plan:
        return plan.fit_coeffs(xs.contiguous(), ts.contiguous(), n_train=n_train, max_iter=max_iter, coeffs0=coeffs0,
                               common_phase=common_phase)
