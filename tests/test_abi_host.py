"""Host-side checks of the C ABI (no GPU): every declared symbol is exported, the
planner's geometry and step table agree with the oracle's, invalid arguments are
rejected with the documented codes before any CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
from oracle import fiber
from paper_1507_00921_gb300 import _lib, describe
from paper_1507_00921_gb300._lib import DBPError

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FS = synth.SAMPLE_RATE


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(dbp_\w+)\s*\(", text, flags=re.M):
                names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_functions()
    assert "dbp_run" in names and "dbp_plan" in names and len(names) >= 9
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.dbp_version().startswith(b"libdbp")


@pytest.mark.parametrize("n_spans,ns,nc,fft", [(10, 1, 8, 1024), (10, 20, 0, 1024), (40, 1, 32, 4096),
                                               (40, 20, 0, 4096), (40, 3, 16, 8192), (40, 4, 32, 8192)])
def test_plan_matches_oracle_step_table(n_spans, ns, nc, fft):
    link = synth.link(n_spans)
    n = 2 ** 15
    info = describe(link, FS, n, method="essfm" if nc else "ssfm", n_steps=ns, n_taps=nc, fft_size=fft)
    cfg = fiber.make_config(link, FS, ns, nc, fft)
    assert info.overlap == cfg.overlap
    assert info.valid == fft - cfg.overlap
    assert info.n_blocks == -(-n // info.valid)
    assert np.allclose(info.step_dz, cfg.dz, rtol=1e-14, atol=0)
    assert np.allclose(info.step_gamma_eff, cfg.gamma_eff, rtol=1e-12, atol=0)
    assert abs(info.beta2 - cfg.beta2) < 1e-12 * abs(cfg.beta2)


def test_plan_nonuniform_steps_and_overrides():
    link = synth.link(40)
    dz = np.array([1e6, 0.2e6, 2e6])
    info = describe(link, FS, 4096, method="essfm", n_steps=3, n_taps=4, step_len_m=dz, fft_size=4096)
    cfg = fiber.make_config(link, FS, 3, 4, 4096, step_len_m=dz)
    assert np.allclose(info.step_gamma_eff, cfg.gamma_eff, rtol=1e-12)
    info = describe(link, FS, 4096, method="essfm", n_steps=3, n_taps=4, gamma_eff=[1.0, 2.0, 3.0],
                    overlap=2048, fft_size=4096)
    assert list(info.step_gamma_eff) == [1.0, 2.0, 3.0] and info.overlap == 2048


@pytest.mark.parametrize("kw,code", [
    (dict(fft_size=1000), _lib.DBP_ERR_INFEASIBLE),
    (dict(fft_size=16384), _lib.DBP_ERR_INFEASIBLE),
    (dict(fft_size=1024, n_spans=40), _lib.DBP_ERR_INFEASIBLE),     # overlap 1432 >= N
    (dict(overlap=4096), _lib.DBP_ERR_INFEASIBLE),
    (dict(overlap=6), _lib.DBP_ERR_ARG),
    (dict(method="ssfm", n_taps=3), _lib.DBP_ERR_ARG),
    (dict(n_taps=65), _lib.DBP_ERR_ARG),
    (dict(n_steps=0), _lib.DBP_ERR_ARG),
    (dict(n_samples=0), _lib.DBP_ERR_ARG),
    (dict(n_waveforms=0), _lib.DBP_ERR_ARG),
    (dict(n_pols=3), _lib.DBP_ERR_ARG),
    (dict(n_pols=1, precision="split_bf16", dft_block=128, fft_size=2048), _lib.DBP_ERR_UNSUPPORTED),
])
def test_invalid_arguments_rejected(kw, code):
    kw = dict(kw)
    link = synth.link(kw.pop("n_spans", 10))
    n = kw.pop("n_samples", 4096)
    args = dict(method="essfm", n_steps=1, n_taps=8, fft_size=4096)
    args.update(kw)
    with pytest.raises(DBPError) as e:
        describe(link, FS, n, **args)
    assert e.value.code == code


def test_null_arguments_and_strerror():
    lib = _lib.load()
    assert lib.dbp_run(None, None, None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_run_host(None, None, None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_plan_get_info(None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_set_coeffs(None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_plan(None, None, None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_grad(None, None, None, None, None, None, None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_set_steps(None, None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_batch_create(None, None, None, 0, 0, 0, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_batch_run(None, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_batch_publish(None, 0, None) == _lib.DBP_ERR_ARG
    assert lib.dbp_batch_status(None) == _lib.DBP_ERR_ARG
    assert lib.dbp_fit_coeffs(None, None, None, 0, 10, 0.0, None, None, None, None, None) == _lib.DBP_ERR_ARG
    lib.dbp_batch_destroy(None)
    lib.dbp_destroy(None)
    for code in range(-9, 1):
        assert lib.dbp_strerror(code) not in (b"", b"unknown error")
    assert lib.dbp_strerror(-99) == b"unknown error"
    info = _lib.dbp_plan_info()
    assert lib.dbp_plan_describe(None, None, None, C.byref(info), None, None) == _lib.DBP_ERR_ARG


def test_block_length_zero_takes_the_section_iii_optimum():
    """fft_size = 0: the planner picks the supported block length that minimises the
    operation count per output sample of Section III, N (8 log2 N + 21 + N_c) / (N - O),
    among those above the overlap (host only, no GPU)."""
    import synth
    from paper_1507_00921_gb300 import complexity, describe
    fs = synth.SAMPLE_RATE
    for spans, method, ns, nc in [(40, "essfm", 1, 32), (10, "essfm", 1, 8), (40, "ssfm", 20, 0), (2, "ssfm", 3, 0),
                                  (20, "essfm", 2, 16), (40, "ffe", 1, 0)]:
        info = describe(synth.link(spans), fs, 1 << 16, method=method, n_steps=ns, n_taps=nc, fft_size=0)
        o = info.overlap
        cands = [n for n in (512, 1024, 2048, 4096, 8192) if n > o]
        cost = {n: complexity.mults_per_sample(n, o, nc, ffe=method == "ffe") for n in cands}
        assert info.fft_size == min(cost, key=cost.get), (spans, method, info.fft_size, cost)
        assert info.valid == info.fft_size - o
    # N = 8M is near-optimal in Section III; at 3200 km (M ~ 1368) that is the largest length
    assert describe(synth.link(40), fs, 1 << 16, method="essfm", n_taps=32, fft_size=0).fft_size == 8192


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU or oracle fallback: with the shared library absent (and no build allowed),
    loading the binding raises instead of computing anything another way."""
    from paper_1507_00921_gb300 import build as _build
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing" / "libdbp.so"))
    with pytest.raises(RuntimeError, match="libdbp not built"):
        _lib.load(build_if_needed=False)
