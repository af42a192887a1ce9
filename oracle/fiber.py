"""Fibre parameters, effective lengths, step table and overlap rule (oracle, float64).

Readings of the paper used here:

* beta2 = -D lambda^2 / (2 pi c); the paper quotes |beta2| = 21 ps^2/km (Section III,
  Fig. 2 discussion) and D is given in ps/(nm km).  lambda is not given: 1550 nm.
* alpha in 1/m from dB/km: alpha = a_dB ln(10)/10 / 1000 (power attenuation).
* Effective length of a step of one span, Section II after Eq. 2:
  dz_eff = (1 - exp(-alpha dz)) / alpha.  For a step that covers several spans or
  part of one (the 20-step SSFM covers four spans per step, the single-step ESSFM the
  whole link, Section IV) the paper is silent; the reading is the integral of the
  forward power profile exp(-alpha (z - z_span_start)) over the step, which reduces
  to the formula above for a one-span step.
* Steps run backwards from the receiver: step 0 covers the last dz_0 metres of the
  link, step s covers [L - sum_{i<=s} dz_i, L - sum_{i<s} dz_i].
* gamma_eff_s = gamma * manakov_factor * dz_eff_s (the Manakov 8/9 factor is not
  stated in Section II; it is a parameter, default 8/9, 1 in most tests).
* Channel memory, Section III: M ~= 2 pi |beta2| L B^2 samples with B equal to the
  sampling rate.  Overlap: O = ceil(M) + 2 N_s N_c (dispersion spread plus the
  N_c-sample reach of the ESSFM filter on each side, per step), rounded up to a
  multiple of 8; the discarded samples are split O/2 at each block end.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0          # m/s
H_PLANCK = 6.62607015e-34      # J s


def beta2_from_D(D_ps_per_nm_km: float, lambda_m: float) -> float:
    """Group-velocity dispersion beta2 [s^2/m] from the dispersion parameter D."""
    D = D_ps_per_nm_km * 1e-12 / (1e-9 * 1e3)          # s/m^2
    return -D * lambda_m ** 2 / (2.0 * math.pi * C_LIGHT)


def alpha_per_m(alpha_db_per_km: float) -> float:
    """Power attenuation coefficient [1/m] from dB/km."""
    return alpha_db_per_km * math.log(10.0) / 10.0 / 1e3


def effective_length(alpha: float, dz: float) -> float:
    """Section II (after Eq. 2): dz_eff = (1 - exp(-alpha dz)) / alpha."""
    if alpha == 0.0:
        return dz
    return (1.0 - math.exp(-alpha * dz)) / alpha


def profile_integral(alpha: float, span_len: float, a: float, b: float) -> float:
    """Integral over [a, b] (metres from the transmitter) of the forward power profile
    exp(-alpha (z - z_span_start(z))), piecewise over spans."""
    if b <= a:
        return 0.0
    total = 0.0
    j0 = int(math.floor(a / span_len))
    j1 = int(math.ceil(b / span_len))
    for j in range(j0, j1):
        s0 = j * span_len
        lo = max(a, s0)
        hi = min(b, s0 + span_len)
        if hi <= lo:
            continue
        total += effective_length(alpha, hi - s0) - effective_length(alpha, lo - s0)
    return total


def channel_memory(beta2: float, length_m: float, bandwidth_hz: float) -> float:
    """Section III: M ~= 2 pi |beta2| L B^2 (samples)."""
    return 2.0 * math.pi * abs(beta2) * length_m * bandwidth_hz ** 2


def overlap_rule(memory: float, n_steps: int, n_taps: int) -> int:
    """O = ceil(M) + 2 N_s N_c, rounded up to a multiple of 8."""
    o = int(math.ceil(memory - 1e-9)) + 2 * n_steps * n_taps
    return ((o + 7) // 8) * 8


@dataclass
class DBPConfig:
    """Everything the overlap-save DBP computes with (float64)."""
    beta2: float                    # s^2/m
    fs: float                       # Hz
    fft_size: int                   # N
    overlap: int                    # O (even)
    dz: np.ndarray                  # [N_s] step lengths (m), step 0 next to the receiver
    gamma_eff: np.ndarray           # [N_s] gamma * manakov * dz_eff (1/W)
    coeffs: np.ndarray              # [N_s, N_c + 1] real ESSFM coefficients c_0..c_Nc
    boundary: str = "periodic"      # or "zero"
    essfm: bool = True              # False: Eq. 2 (SSFM) nonlinear sub-step

    @property
    def n_steps(self) -> int:
        return len(self.dz)

    @property
    def n_taps(self) -> int:
        return self.coeffs.shape[1] - 1


def step_table(link: dict, n_steps: int, step_len_m=None):
    """Backward step lengths dz_s and gamma_eff_s for a link (see module docstring)."""
    L = link["n_spans"] * link["span_len_m"]
    alpha = alpha_per_m(link["alpha_db_per_km"])
    if step_len_m is None:
        dz = np.full(n_steps, L / n_steps)
    else:
        dz = np.asarray(step_len_m, dtype=np.float64)
    gamma = link["gamma_per_W_km"] * 1e-3 * link.get("manakov_factor", 1.0)
    geff = np.empty(n_steps)
    top = L
    for s in range(n_steps):
        bot = top - dz[s]
        geff[s] = gamma * profile_integral(alpha, link["span_len_m"], bot, top)
        top = bot
    return dz, geff


def make_config(link: dict, fs: float, n_steps: int, n_taps: int, fft_size: int,
                coeffs=None, overlap=None, boundary="periodic", essfm=None,
                step_len_m=None, gamma_eff=None) -> DBPConfig:
    """Assemble a DBPConfig the way the backpropagation plan is defined."""
    beta2 = beta2_from_D(link["D_ps_per_nm_km"], link["lambda_m"])
    dz, geff = step_table(link, n_steps, step_len_m)
    if gamma_eff is not None:
        geff = np.asarray(gamma_eff, dtype=np.float64)
    if coeffs is None:
        c = np.zeros((n_steps, n_taps + 1))
        c[:, 0] = 1.0
    else:
        c = np.asarray(coeffs, dtype=np.float64)
        if c.ndim == 1:
            c = np.tile(c, (n_steps, 1))
    if overlap is None:
        L = float(np.sum(dz))
        overlap = overlap_rule(channel_memory(beta2, L, fs), n_steps, n_taps)
    if essfm is None:
        essfm = n_taps > 0
    return DBPConfig(beta2=beta2, fs=fs, fft_size=fft_size, overlap=int(overlap), dz=dz,
                     gamma_eff=geff, coeffs=c, boundary=boundary, essfm=essfm)


def per_step_configs(link: dict, fs: float, n_steps: int, n_taps: int, fft_size: int, coeffs=None,
                     boundary="periodic", essfm=None, step_len_m=None, overlap=None, ffe=False):
    """One single-step DBPConfig per step for the per-step-pass scheme: step s is its own
    overlap-and-save pass with overlap ceil(M_s) + 2 N_c (M_s the memory of that step's
    length, Section III), rounded up to a multiple of 8, unless ``overlap`` is given."""
    full = make_config(link, fs, n_steps, n_taps, fft_size, coeffs=coeffs, overlap=1 << 30, boundary=boundary,
                       essfm=essfm, step_len_m=step_len_m, gamma_eff=np.zeros(n_steps) if ffe else None)
    cfgs = []
    for s in range(n_steps):
        o = overlap if overlap else overlap_rule(channel_memory(full.beta2, float(full.dz[s]), fs), 1, n_taps)
        cfgs.append(DBPConfig(beta2=full.beta2, fs=fs, fft_size=fft_size, overlap=int(o), dz=full.dz[s:s + 1],
                              gamma_eff=full.gamma_eff[s:s + 1], coeffs=full.coeffs[s:s + 1], boundary=boundary,
                              essfm=full.essfm))
    return cfgs
