"""One-polarization DBP (the scalar SSFM / ESSFM that Eq. 3 extends to PM signals):
the CUDA path, which carries two consecutive blocks in the two polarization lanes of a
CTA, against (i) the dual-polarization path with the second polarization zero (same
FP32 arithmetic, so bit-identical) and (ii) the FP64 oracle run on [1, n] waveforms."""
import numpy as np
import pytest

import synth
from oracle import dbp as odbp
from oracle import fiber
from oracle import link as olink

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE
TOL_RMS = 1e-5
TOL_MAX = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def scalar_rx(n_sym, spans, seed, dbm=2.0):
    """One polarization of a PM-QPSK waveform through a scalar link (manakov_factor 1)."""
    link = synth.link(spans, manakov_factor=1.0)
    tx, _, _ = synth.pm_qpsk_waveform(n_sym, seed, dbm)
    r = olink.forward(tx[:1], link, FS, steps_per_span=20, ase_seed=seed + 1)
    return link, r


CASES = [
    ("essfm1_nc8_N1024", 10, 2 ** 13, dict(method="essfm", n_steps=1, n_taps=8, fft_size=1024)),
    ("ssfm8_N2048_zero", 10, 2 ** 13 + 77, dict(method="ssfm", n_steps=8, fft_size=2048, boundary="zero")),
    ("ffe_N512", 10, 2 ** 12, dict(method="ffe", n_steps=1, fft_size=512)),
    ("essfm2_nc16_N4096_3wave", 40, 2 ** 14 + 5, dict(method="essfm", n_steps=2, n_taps=16, fft_size=4096,
                                                      n_waveforms=3)),
    ("essfm1_nc32_N8192", 40, 2 ** 15, dict(method="essfm", n_steps=1, n_taps=32, fft_size=8192)),
    ("ssfm4_per_step_N1024", 20, 2 ** 13, dict(method="ssfm", n_steps=4, fft_size=1024, scheme="per_step")),
]


@pytest.mark.parametrize("name,spans,n_sym,kw", CASES, ids=[c[0] for c in CASES])
def test_single_pol_equals_dual_pol_with_zero_second_pol_and_oracle(torch_cuda, name, spans, n_sym, kw):
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    kw = dict(kw)
    nw = kw.pop("n_waveforms", 1)
    rs = []
    for w in range(nw):
        link, r = scalar_rx(n_sym // 2, spans, synth.BASE_SEED + 1200 + 10 * w)
        rs.append(r)
    x1 = np.stack(rs).astype(np.complex64)                       # [nw, 1, n]
    n = x1.shape[-1]
    x2 = np.concatenate([x1, np.zeros_like(x1)], axis=1)         # [nw, 2, n]
    with Plan(link, FS, n, n_waveforms=nw, n_pols=1, **kw) as p1, \
            Plan(link, FS, n, n_waveforms=nw, n_pols=2, **kw) as p2:
        assert p1.info.n_blocks == p2.info.n_blocks
        y1 = p1.run(torch.from_numpy(x1).cuda()).cpu().numpy()
        y2 = p2.run(torch.from_numpy(x2).cuda()).cpu().numpy()
        h1 = p1.run_host(torch.from_numpy(x1)).numpy()
        info = p1.info
    np.testing.assert_array_equal(y1[:, 0], y2[:, 0])
    np.testing.assert_array_equal(h1, y1)
    assert not np.any(y2[:, 1])

    method = kw.get("method", "essfm")
    nc = kw.get("n_taps", 0)
    ns = kw.get("n_steps", 1)
    ref_in = x1.astype(np.complex128)
    if kw.get("scheme") == "per_step":
        cfgs = fiber.per_step_configs(link, FS, ns, nc, kw["fft_size"], boundary=kw.get("boundary", "periodic"),
                                      essfm=method == "essfm", ffe=method == "ffe")
        ref = odbp.dbp_per_step(ref_in, cfgs)
    else:
        cfg = fiber.make_config(link, FS, ns, nc, kw["fft_size"], overlap=info.overlap,
                                boundary=kw.get("boundary", "periodic"), essfm=method == "essfm",
                                gamma_eff=np.zeros(ns) if method == "ffe" else None)
        ref = odbp.dbp(ref_in, cfg)
    err = y1.astype(np.complex128) - ref
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    rel_rms = np.sqrt(np.mean(np.abs(err) ** 2)) / rms
    max_rel = np.max(np.abs(err)) / rms
    print(f"\n{name}: {info.n_blocks} blocks, rel RMS {rel_rms:.2e}, max {max_rel:.2e}")
    assert rel_rms <= TOL_RMS and max_rel <= TOL_MAX


def test_single_pol_unsupported_calls(torch_cuda):
    torch = torch_cuda
    from paper_1507_00921_gb300 import Batch, DBPError, Plan
    link = synth.link(10, manakov_factor=1.0)
    n = 4096
    x = (torch.randn(1, n, dtype=torch.complex64, device="cuda") * 0.03).contiguous()
    with Plan(link, FS, n, n_pols=1, method="essfm", n_steps=1, n_taps=4, fft_size=1024) as plan:
        with pytest.raises(DBPError) as ei:
            plan.grad(x, x)
        assert ei.value.code == -7
        with pytest.raises(DBPError) as ei:
            plan.fit_coeffs(x, x)
        assert ei.value.code == -7
        with pytest.raises(DBPError) as ei:
            Batch([plan], [x], [torch.empty_like(x)])
        assert ei.value.code == -7
