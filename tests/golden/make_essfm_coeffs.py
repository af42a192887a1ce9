"""Writes tests/golden/essfm_coeffs.json: ESSFM coefficients fitted by the FP64 oracle.

Section IV: the coefficients minimise the MSE between the ESSFM output and the output
of an SSFM with several steps per span, on a training waveform.  Here the training
waveform is a separate seeded PM-QPSK waveform through the oracle's link simulator
(with ASE); the target is a 4-steps-per-span SSFM backpropagation of it.  Only the
oracle and the input generators are used.  Run: python tests/golden/make_essfm_coeffs.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import dbp as odbp  # noqa: E402
from oracle import fiber, fit  # noqa: E402
from oracle import link as olink  # noqa: E402

CASES = {
    # name: spans, n_symbols, dBm, N_c, fft, forward steps/span
    "800km_nc8_N1024_2dBm": (10, 2 ** 14, 2.0, 8, 1024, 100),
    "3200km_nc32_N4096_2dBm": (40, 2 ** 14, 2.0, 32, 4096, 25),
    "3200km_nc16_N4096_2dBm": (40, 2 ** 14, 2.0, 16, 4096, 25),
}


def main():
    out = {"_source": "fitted by tests/golden/make_essfm_coeffs.py with the FP64 oracle "
                      "(Section IV: MSE against a multi-step-per-span SSFM output)"}
    for name, (spans, nsym, dbm, nc, fft, sps) in CASES.items():
        link = synth.link(spans)
        tx, _, _ = synth.pm_qpsk_waveform(nsym, synth.BASE_SEED + 500 + spans, dbm)
        r = olink.forward(tx, link, synth.SAMPLE_RATE, steps_per_span=sps, ase_seed=synth.BASE_SEED + 600 + spans)
        tcfg = fiber.make_config(link, synth.SAMPLE_RATE, 4 * spans, 0, fft)
        target = odbp.dbp(r, tcfg)
        cfg = fiber.make_config(link, synth.SAMPLE_RATE, 1, nc, fft)
        c = fit.fit_single_step(r, target, cfg)
        out[name] = {"n_taps": nc, "fft_size": fft, "n_spans": spans, "launch_dbm": dbm,
                     "coeffs": [float(v) for v in c]}
        print(name, np.round(c[:6], 4))
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "essfm_coeffs.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
