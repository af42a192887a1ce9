"""Block-length autotuner for the overlap-save DBP.

Section III of arXiv:1507.00921 chooses the block length N by minimising the operation
count per sample, N(8 log2 N + 21 + N_c)/(N - M), and finds N = 8M near-optimal for its
hardware-agnostic count.  On the GPU the optimum also depends on occupancy and shared
memory, so the tuner uses that count only as a prior (to order and prune candidates)
and times the feasible candidates on the device, with the plan's own overlap rule.
Results are cached per (link, method, steps, taps, sample rate).
"""
from __future__ import annotations

from . import complexity
from .dbp import Plan, describe

SIZES = (512, 1024, 2048, 4096, 8192)
_cache: dict = {}


def candidates(link: dict, fs: float, method: str, n_steps: int, n_taps: int, max_candidates: int = 3):
    """Feasible block lengths (overlap < N), ordered by the Section III operation count."""
    out = []
    for n in SIZES:
        try:
            info = describe(link, fs, 1 << 16, method=method, n_steps=n_steps, n_taps=n_taps, fft_size=n)
        except Exception:
            continue
        cost = complexity.total_mults(n, info.overlap, n_steps, n_taps if method == "essfm" else 0)
        out.append((cost, n))
    out.sort()
    return [n for _, n in out[:max_candidates]]


def tune(link: dict, fs: float, method: str, n_steps: int, n_taps: int, n_samples: int = 1 << 19,
         n_waveforms: int = 8, reps: int = 5) -> int:
    """Fastest block length for this configuration, timed with CUDA events."""
    import torch
    key = (tuple(sorted(link.items())), float(fs), method, int(n_steps), int(n_taps))
    if key in _cache:
        return _cache[key]
    cands = candidates(link, fs, method, n_steps, n_taps)
    if not cands:
        raise ValueError("no feasible block length for this link")
    x = torch.randn(n_waveforms, 2, n_samples, dtype=torch.complex64, device="cuda") * 0.03
    y = torch.empty_like(x)
    best = None
    for n in cands:
        with Plan(link, fs, n_samples, n_waveforms=n_waveforms, method=method, n_steps=n_steps, n_taps=n_taps,
                  fft_size=n) as plan:
            plan.run(x, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                plan.run(x, y)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
        if best is None or t < best[1]:
            best = (n, t)
    _cache[key] = best[0]
    return best[0]
