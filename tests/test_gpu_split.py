"""Split-precision linear sub-step (DFT-matrix GEMMs on the tensor cores, hi/lo split
BF16 or FP16 operands, FP32 accumulation) against the FP64 oracle.

Tolerances from the arithmetic: an FP16 hi + lo pair carries ~22 significant bits
(error ~2^-22 per operand, below FP32 rounding of the accumulation), so the FP32 bar
(relative RMS 1e-5) applies; a BF16 pair carries ~16 bits (~2^-17 rounding per
operand, 1.5e-5 at worst for one product term, averaging down over the N_a-term sums),
measured 4.8e-6 to 9.5e-6 on these cases, so relative RMS 2e-5 (about twice the worst
measured)."""
import numpy as np
import pytest

import synth
from oracle import dbp as odbp
from oracle import fiber
from oracle import link as olink
from oracle import rx

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE
TOL = {"split_fp16": 1e-5, "split_bf16": 2e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def coeffs(nc):
    c = 0.6 * np.exp(-np.arange(nc + 1) / 6.0)
    return (c / (c[0] + 2 * c[1:].sum())).astype(np.float32)


# N_a = 64 with N = 1024 / 2048 runs on tcgen05 (tensor memory accumulators); the other
# sizes on mma.sync
CASES = [(prec, fft, na, spans, ns, nc)
         for prec in ("split_fp16", "split_bf16")
         for (fft, na, spans, ns, nc) in [(1024, 64, 10, 1, 16), (1024, 128, 10, 1, 16), (1024, 256, 10, 1, 16),
                                          (2048, 128, 20, 2, 8), (4096, 256, 40, 1, 32), (2048, 64, 10, 3, 0),
                                          (2048, 64, 20, 2, 32), (1024, 64, 10, 4, 8)]]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}_N{c[1]}_NA{c[2]}_{c[3] * 80}km_ns{c[4]}_nc{c[5]}" for c in CASES])
def test_split_precision_against_oracle(torch_cuda, case):
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    prec, fft, na, spans, ns, nc = case
    link = synth.link(spans)
    n = 3 * fft + 77
    x = synth.random_field(2, n, synth.dbm_to_w(2.0), seed=fft + na).astype(np.complex64)
    c = coeffs(nc) if nc else None
    method = "essfm" if nc else "ssfm"
    with Plan(link, FS, n, n_waveforms=2, method=method, n_steps=ns, n_taps=nc, coeffs=c, fft_size=fft,
              precision=prec, dft_block=na) as plan:
        got = plan.run(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
        ov = plan.info.overlap
        assert plan.status() == 0
    cfg = fiber.make_config(link, FS, ns, nc, fft, coeffs=None if c is None else c.astype(np.float64), overlap=ov,
                            essfm=nc > 0)
    ref = odbp.dbp(x.astype(np.complex128), cfg)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\n{prec} N={fft} N_a={na} {spans * 80} km N_s={ns} N_c={nc}: relative RMS {rel:.3e}")
    assert rel <= TOL[prec], rel


def test_split_precision_q_factor(torch_cuda):
    """Q-factor per path on an 800 km link waveform (config-3 shape: N_s = 1, N_c = 16)."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    link = synth.link(10)
    tx, sym, bits = synth.pm_qpsk_waveform(2 ** 14, synth.BASE_SEED + 300, 2.0)
    r = olink.forward(tx, link, FS, steps_per_span=50, ase_seed=synth.BASE_SEED + 301).astype(np.complex64)
    c = coeffs(16)
    q = {}
    for prec, na in [("fp32", 0), ("split_fp16", 64), ("split_bf16", 64), ("split_bf16", 256)]:
        with Plan(link, FS, r.shape[-1], method="essfm", n_steps=1, n_taps=16, coeffs=c, fft_size=1024,
                  precision=prec, dft_block=na) as plan:
            out = plan.run(torch.from_numpy(r[None]).cuda()).cpu().numpy()[0].astype(np.complex128)
        q[(prec, na)] = rx.evaluate(out, sym, bits)["q_db"]
    cfg = fiber.make_config(link, FS, 1, 16, 1024, coeffs=c.astype(np.float64))
    q_ref = rx.evaluate(odbp.dbp(r.astype(np.complex128), cfg), sym, bits)["q_db"]
    print("\nQ (dB): oracle %.3f, " % q_ref + ", ".join(f"{k[0]}/{k[1]} {v:.3f}" for k, v in q.items()))
    assert abs(q[("fp32", 0)] - q_ref) <= 0.05
    assert abs(q[("split_fp16", 64)] - q_ref) <= 0.05
    assert abs(q[("split_bf16", 64)] - q_ref) <= 0.05


@pytest.mark.parametrize("prec", ["split_fp16", "split_bf16"])
def test_tcgen05_and_mma_sync_paths_agree(torch_cuda, prec, monkeypatch):
    """The tcgen05 kernel (N_a = 64) and the warp-level mma.sync kernel compute the same
    split products in different orders: outputs agree to the split's own precision, over
    several blocks per tile, ragged tails, zero boundary, one and two steps."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    link = synth.link(10)
    n = 5 * 1024 + 333
    x = torch.from_numpy(synth.random_field(3, n, synth.dbm_to_w(3.0), seed=41).astype(np.complex64)).cuda()
    outs = []
    for legacy in ("0", "1"):
        monkeypatch.setenv("DBP_SPLIT_MMA_SYNC", legacy)
        with Plan(link, FS, n, n_waveforms=3, method="essfm", n_steps=2, n_taps=8, coeffs=coeffs(8),
                  fft_size=1024, precision=prec, dft_block=64, boundary="zero") as plan:
            outs.append(plan.run(x).cpu().numpy().astype(np.complex128))
            assert plan.status() == 0
    rel = np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1])
    assert rel <= TOL[prec], rel


@pytest.mark.parametrize("prec", ["split_fp16", "split_bf16"])
@pytest.mark.parametrize("kind", ["nonuniform_steps", "ffe", "ssfm_zero"])
def test_tcgen05_path_step_tables_and_methods(torch_cuda, prec, kind):
    """The tcgen05 kernel's per-step H tables (unequal step lengths), the linear-only
    method (FFE) and the SSFM with zero boundary against the FP64 oracle."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    link = synth.link(20)
    n = 4 * 2048 + 301
    x = synth.random_field(2, n, synth.dbm_to_w(2.0), seed=97).astype(np.complex64)
    kw = {"nonuniform_steps": dict(method="essfm", n_steps=3, n_taps=8, coeffs=coeffs(8),
                                   step_len_m=np.array([0.4e6, 0.7e6, 0.5e6])),
          "ffe": dict(method="ffe", n_steps=1),
          "ssfm_zero": dict(method="ssfm", n_steps=4, boundary="zero")}[kind]
    with Plan(link, FS, n, n_waveforms=2, fft_size=2048, precision=prec, dft_block=64, **kw) as plan:
        got = plan.run(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
        ov = plan.info.overlap
        assert plan.status() == 0
    c = kw.get("coeffs")
    nc = kw.get("n_taps", 0)
    cfg = fiber.make_config(link, FS, kw["n_steps"], nc, 2048, coeffs=None if c is None else c.astype(np.float64),
                            overlap=ov, boundary=kw.get("boundary", "periodic"), essfm=kw["method"] == "essfm",
                            step_len_m=kw.get("step_len_m"),
                            gamma_eff=np.zeros(1) if kw["method"] == "ffe" else None)
    ref = odbp.dbp(x.astype(np.complex128), cfg)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\ntcgen05 {prec} {kind}: relative RMS {rel:.3e}")
    assert rel <= TOL[prec], rel
