"""Block-length and overlap autotuner for the overlap-save DBP.

Section III of arXiv:1507.00921 chooses the block length N by minimising the operation
count per sample, N(8 log2 N + 21 + N_c)/(N - M), and finds N = 8M near-optimal for its
hardware-agnostic count; the overlap must be at least the channel memory M (plus the
ESSFM filter's reach, 2 N_s N_c, in this implementation).  On the GPU the optimum also
depends on occupancy and shared memory, so the tuner uses that count only as a prior
(to order and prune block lengths) and times candidates (N, O) on the device:

* O_min, the plan's own rule (ceil(M) + 2 N_s N_c rounded up to a multiple of 8);
* O_same, the largest overlap that keeps the number of blocks of O_min for the tuning
  length (so the same work, and a wider margin against the dispersion tails);
* O_min + (N - O_min) / 8 rounded to 8, a costlier point.

The choice is the fastest candidate; among candidates within ``tie`` (relative) of the
fastest time, the one with the largest overlap.  Results are cached per (link, method,
steps, taps, sample rate, tuning length, waveforms).
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import complexity
from .dbp import Plan, describe

SIZES = (512, 1024, 2048, 4096, 8192)
_cache: dict = {}


@dataclass
class Choice:
    fft_size: int
    overlap: int
    min_overlap: int                      # the rule's overlap for this block length
    timings: dict = field(default_factory=dict)   # (N, O) -> ms per launch


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


def overlap_candidates(fft_size: int, o_min: int, n_samples: int):
    """Overlaps to time for one block length (multiples of 8 in [o_min, N))."""
    nb = -(-n_samples // (fft_size - o_min))
    o_same = fft_size - (-(-n_samples // nb))          # largest O with ceil(n / (N - O)) == nb
    o_same -= o_same % 8
    o_wide = o_min + (fft_size - o_min) // 8
    o_wide -= o_wide % 8
    out = [o_min]
    for o in (o_same, o_wide):
        if o_min < o < fft_size and o not in out:
            out.append(o)
    return out


def tune(link: dict, fs: float, method: str, n_steps: int, n_taps: int, n_samples: int = 1 << 19,
         n_waveforms: int = 8, reps: int = 5, tie: float = 0.01) -> Choice:
    """Fastest (block length, overlap) for this configuration, timed with CUDA events."""
    import torch
    key = (tuple(sorted(link.items())), float(fs), method, int(n_steps), int(n_taps), int(n_samples),
           int(n_waveforms))
    if key in _cache:
        return _cache[key]
    sizes = candidates(link, fs, method, n_steps, n_taps)
    if not sizes:
        raise ValueError("no feasible block length for this link")
    x = torch.randn(n_waveforms, 2, n_samples, dtype=torch.complex64, device="cuda") * 0.03
    y = torch.empty_like(x)
    timings, o_mins = {}, {}
    for n in sizes:
        o_min = describe(link, fs, n_samples, method=method, n_steps=n_steps, n_taps=n_taps, fft_size=n).overlap
        o_mins[n] = o_min
        for o in overlap_candidates(n, o_min, n_samples):
            with Plan(link, fs, n_samples, n_waveforms=n_waveforms, method=method, n_steps=n_steps,
                      n_taps=n_taps, fft_size=n, overlap=o) as plan:
                plan.run(x, y)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    plan.run(x, y)
                e1.record()
                e1.synchronize()
                timings[(n, o)] = e0.elapsed_time(e1) / reps
    choice = pick(timings, tie)
    best = Choice(choice[0], choice[1], o_mins[choice[0]], timings)
    _cache[key] = best
    return best


def pick(timings: dict, tie: float = 0.01):
    """The (N, O) of ``timings`` with the smallest time; among those within ``tie`` of it,
    the largest overlap (then the smaller block length)."""
    t_best = min(timings.values())
    near = [k for k, t in timings.items() if t <= t_best * (1.0 + tie)]
    return max(near, key=lambda k: (k[1], -k[0]))
