"""Equal-Q comparison on a synthetic 3200 km link (Section IV's question: how many SSFM
steps does one ESSFM step replace?).  The CUDA path backpropagates a received test
waveform (oracle link simulator with ASE, 2 dBm per polarization) with linear-only
compensation (FFE), with SSFM for N_s = 1..40, and with single-step ESSFM whose
coefficients are fitted on the GPU (dbp_fit_coeffs, Section IV: minimum MSE against a
160-step SSFM output of a separate training waveform, with and without a common phase
fitted alongside).  The Q table is printed.  The checks are facts that hold by
construction or are robust: SSFM improves with the step count, and the fit with a
common phase, whose feasible set contains the linear-only compensation, is not worse
than FFE."""
import numpy as np
import pytest

import synth
from oracle import link as olink
from oracle import rx

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE
SPANS, FWD_STEPS, DBM, FFT = 40, 25, 2.0, 8192
STEPS = (1, 2, 4, 10, 20, 40)


def test_essfm_single_step_against_ssfm_step_counts():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_00921_gb300 import Plan
    from paper_1507_00921_gb300.fit import fit_gauss_newton
    link = synth.link(SPANS)
    waves = {}
    for name, seed in (("train", 1400), ("test", 1500)):
        tx, sym, bits = synth.pm_qpsk_waveform(2 ** 14, synth.BASE_SEED + seed, DBM)
        r = olink.forward(tx, link, FS, steps_per_span=FWD_STEPS, ase_seed=synth.BASE_SEED + seed + 1)
        waves[name] = (torch.from_numpy(r.astype(np.complex64)).cuda(), sym, bits)
    n = waves["test"][0].shape[-1]

    def run(x, **kw):
        with Plan(link, FS, n, fft_size=FFT, **kw) as plan:
            return plan.run(x[None].contiguous())[0]

    def q_of(y):
        return rx.evaluate(y.cpu().numpy().astype(np.complex128), waves["test"][1], waves["test"][2])["q_db"]

    xt = waves["test"][0]
    q = {"ffe": q_of(run(xt, method="ffe", n_steps=1))}
    for ns in STEPS:
        q[f"ssfm{ns}"] = q_of(run(xt, method="ssfm", n_steps=ns))
    target = run(waves["train"][0], method="ssfm", n_steps=160)
    for nc in (8, 32):
        c, _ = fit_gauss_newton(link, FS, waves["train"][0], target, nc, FFT)
        q[f"essfm1_nc{nc}"] = q_of(run(xt, method="essfm", n_steps=1, n_taps=nc, coeffs=c.astype(np.float32)))
        c, _, _ = fit_gauss_newton(link, FS, waves["train"][0], target, nc, FFT, common_phase=True)
        q[f"essfm1_nc{nc}_phase"] = q_of(run(xt, method="essfm", n_steps=1, n_taps=nc, coeffs=c.astype(np.float32)))
    print(f"\n3200 km, {DBM} dBm, Q (dB): " + ", ".join(f"{k} {v:.2f}" for k, v in q.items()))
    for key in ("essfm1_nc32", "essfm1_nc32_phase"):
        match = [ns for ns in STEPS if q[f"ssfm{ns}"] >= q[key]]
        print(f"{key}: Q {q[key]:.2f} dB, reached by SSFM with N_s >= {match[0] if match else '> 40'}")
    assert q["ssfm40"] > q["ssfm20"] > q["ssfm10"]
    assert q["essfm1_nc32_phase"] >= q["ffe"] - 0.1
    assert q["essfm1_nc8_phase"] >= q["ffe"] - 0.1
