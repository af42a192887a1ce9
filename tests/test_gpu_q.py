"""Q-factor match: the CUDA path and the FP64 oracle backpropagate the same received
waveform (oracle link simulator with ASE); their Q-factors agree within 0.05 dB and
their hard QPSK decisions are identical.  Coefficients: tests/golden/essfm_coeffs.json
(fitted by the oracle on a separate training waveform)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import dbp as odbp
from oracle import fiber
from oracle import link as olink
from oracle import rx

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "essfm_coeffs.json")))

LINKS = {"800km": (10, 100), "3200km": (40, 25)}      # spans, forward steps per span
CASES = [
    ("800km", "essfm", 1, "800km_nc8_N1024_2dBm", 1024),
    ("800km", "ssfm", 20, None, 1024),
    ("3200km", "essfm", 1, "3200km_nc32_N4096_2dBm", 4096),
    ("3200km", "ssfm", 20, None, 4096),
    ("3200km", "essfm", 1, "3200km_nc16_N4096_2dBm", 8192),
]


@pytest.fixture(scope="module")
def received():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = {}
    for name, (spans, sps) in LINKS.items():
        tx, sym, bits = synth.pm_qpsk_waveform(2 ** 14, synth.BASE_SEED + 700 + spans, 2.0)
        r = olink.forward(tx, synth.link(spans), FS, steps_per_span=sps, ase_seed=synth.BASE_SEED + 800 + spans)
        out[name] = (r.astype(np.complex64), sym, bits)
    return out


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}_{c[1]}{c[2]}_N{c[4]}" for c in CASES])
def test_q_and_decisions_match_oracle(received, case):
    import torch
    from paper_1507_00921_gb300 import Plan
    lname, method, ns, cname, fft = case
    spans = LINKS[lname][0]
    link = synth.link(spans)
    r, sym, bits = received[lname]
    nc = GOLD[cname]["n_taps"] if cname else 0
    c = np.asarray(GOLD[cname]["coeffs"], dtype=np.float32) if cname else None
    with Plan(link, FS, r.shape[-1], method=method, n_steps=ns, n_taps=nc, coeffs=c, fft_size=fft) as plan:
        got = plan.run(torch.from_numpy(r[None]).cuda()).cpu().numpy()[0].astype(np.complex128)
        ov = plan.info.overlap
    cfg = fiber.make_config(link, FS, ns, nc, fft, coeffs=None if c is None else c.astype(np.float64),
                            overlap=ov, essfm=(method == "essfm"))
    ref = odbp.dbp(r.astype(np.complex128), cfg)
    eg = rx.evaluate(got, sym, bits)
    eo = rx.evaluate(ref, sym, bits)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\n{lname} {method} N_s={ns} N_c={nc} N={fft}: Q gpu {eg['q_db']:.3f} dB, oracle {eo['q_db']:.3f} dB, "
          f"BER {eg['ber']:.2e}, rel RMS {rel:.2e}")
    assert rel <= 1e-5
    assert abs(eg["q_db"] - eo["q_db"]) <= 0.05
    assert np.array_equal(eg["decisions"], eo["decisions"])
