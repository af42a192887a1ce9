"""Autotuner of the block length N and the overlap O (Section III: N near 8M is
near-optimal for the operation count; O at least the channel memory M).  Host logic on
the CPU; on the GPU, the tuned plan is feasible, is the fastest of the timed candidates
(ties within 1 % go to the wider overlap), and a plan at a non-default overlap matches
the FP64 oracle."""
import numpy as np
import pytest

import synth
from paper_1507_00921_gb300 import autotune, describe

FS = synth.SAMPLE_RATE


def test_overlap_candidates_keep_or_grow_the_block_count():
    for n_fft, o_min, n in [(4096, 1368, 1 << 19), (8192, 1432, 1 << 19), (1024, 344, 5000), (2048, 1368, 777)]:
        cands = autotune.overlap_candidates(n_fft, o_min, n)
        assert cands[0] == o_min
        assert all(o % 8 == 0 and o_min <= o < n_fft for o in cands)
        assert len(set(cands)) == len(cands)
        nb = -(-n // (n_fft - o_min))
        same = [o for o in cands if -(-n // (n_fft - o)) == nb]
        # the widest candidate with the rule's block count is the largest such multiple of 8
        o_same = max(same)
        assert o_same + 8 >= n_fft or -(-n // (n_fft - o_same - 8)) > nb


def test_pick_fastest_with_overlap_tie_break():
    t = {(4096, 1368): 1.00, (4096, 1400): 1.005, (4096, 1800): 1.3, (8192, 1368): 0.95}
    assert autotune.pick(t, tie=0.01) == (8192, 1368)
    t[(8192, 1600)] = 0.955                          # within 1 % of the best: the wider overlap wins
    assert autotune.pick(t, tie=0.01) == (8192, 1600)
    assert autotune.pick(t, tie=0.0) == (8192, 1368)


def test_block_length_candidates_are_feasible():
    link = synth.link(40)
    sizes = autotune.candidates(link, FS, "essfm", 1, 32)
    assert sizes and 512 not in sizes and 1024 not in sizes      # overlap 1432 does not fit
    for n in sizes:
        assert describe(link, FS, 1 << 16, method="essfm", n_steps=1, n_taps=32, fft_size=n).overlap < n


@pytest.mark.gpu
def test_tuned_plan_is_fastest_and_matches_oracle_at_wider_overlap():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import dbp as odbp
    from oracle import fiber
    from paper_1507_00921_gb300 import Plan
    link = synth.link(20)
    ch = autotune.tune(link, FS, "essfm", 1, 16, n_samples=1 << 17, n_waveforms=4, reps=3)
    assert ch.min_overlap <= ch.overlap < ch.fft_size
    assert (ch.fft_size, ch.overlap) in ch.timings and len(ch.timings) >= 3
    t_best = min(ch.timings.values())
    assert ch.timings[(ch.fft_size, ch.overlap)] <= 1.01 * t_best
    assert all(o <= ch.overlap for (nn, o), t in ch.timings.items() if t <= 1.01 * t_best)
    # parity with the oracle at a non-default overlap of the tuned block length
    wide = max(o for (nn, o) in ch.timings if nn == ch.fft_size)
    assert wide > ch.min_overlap
    n = 3 * ch.fft_size + 101
    c = 0.6 * np.exp(-np.arange(17) / 5.0)
    c = (c / (c[0] + 2 * c[1:].sum())).astype(np.float32)
    x = synth.random_field(1, n, synth.dbm_to_w(2.0), seed=33).astype(np.complex64)
    with Plan(link, FS, n, method="essfm", n_steps=1, n_taps=16, coeffs=c, fft_size=ch.fft_size,
              overlap=wide) as plan:
        assert plan.info.overlap == wide
        got = plan.run(torch.from_numpy(x).cuda()).cpu().numpy()[0].astype(np.complex128)
    cfg = fiber.make_config(link, FS, 1, 16, ch.fft_size, coeffs=c.astype(np.float64), overlap=wide)
    ref = odbp.dbp(x[0].astype(np.complex128), cfg)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.sqrt(np.mean(np.abs(got - ref) ** 2)) / rms <= 1e-5
    assert np.max(np.abs(got - ref)) / rms <= 1e-4
