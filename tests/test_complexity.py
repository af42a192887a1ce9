"""The complexity model reproduces the operation counts printed in the paper
(tests/golden/paper_section3_4_numbers.json, each entry with its citation)."""
import json
import os

import pytest

from paper_1507_00921_gb300 import complexity as cx

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_section3_4_numbers.json")))


def test_section_iv_counts():
    g = GOLD["section_IV_real_mults_per_sample"]
    n, m = g["N"], g["M"]
    assert round(cx.mults_per_sample(n, m, ffe=True)) == g["ffe"]
    assert round(cx.total_mults(n, m, 1, 32)) == g["essfm_1step_nc32"]
    assert round(cx.total_mults(n, m, 16)) == g["ssfm_16step"]
    assert round(cx.total_mults(n, m, 20)) == g["ssfm_20step"]


def test_section_iv_reduction_factors():
    g = GOLD["section_IV_real_mults_per_sample"]
    r = GOLD["section_IV_reductions"]
    ratio = cx.total_mults(g["N"], g["M"], 20) / cx.total_mults(g["N"], g["M"], 1, 32)
    assert round(ratio) == r["complexity_factor"]
    assert 20 / 1 == r["latency_factor"]          # cascaded FFT pairs: 20 steps vs 1 (Section III)


def test_section_iii_fig2_ratios():
    g = GOLD["section_III_fig2"]
    m = cx.memory_samples(g["beta2_ps2_per_km"] * 1e-27, g["length_km"] * 1e3, g["bandwidth_hz"])
    n = 8 * m
    e = cx.mults_per_sample(n, m, g["nc"])
    assert e / cx.mults_per_sample(n, m) == pytest.approx(g["essfm_over_ssfm"], abs=g["tolerance"])
    assert e / cx.mults_per_sample(n, m, ffe=True) == pytest.approx(g["essfm_over_ffe"], abs=g["tolerance"])


def test_memory_example():
    g = GOLD["section_III_memory_example"]
    m = cx.memory_samples(g["beta2_ps2_per_km"] * 1e-27, g["length_km"] * 1e3, g["bandwidth_hz"])
    assert m == pytest.approx(g["M"], rel=g["tolerance"])


def test_additions_model():
    assert cx.adds_per_sample(8192, 1024, 32) == pytest.approx(8192 * (104 + 11 + 64) / 7168)
    with pytest.raises(ValueError):
        cx.mults_per_sample(1024, 1024)
