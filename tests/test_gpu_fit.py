"""Fitting ESSFM coefficients with the adjoint (200 Adam iterations on the symbol MSE,
Section IV footnote) over a simulated 3200 km link: the loss falls, and the fitted
filter improves Q on a separate test waveform over the unfitted start (a flat filter
c_i = 1 / (2 N_c + 1), the same total weight as the SSFM's c_0 = 1)."""
import numpy as np
import pytest

import synth
from oracle import link as olink
from oracle import rx

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE


def test_adam_fit_through_adjoint_improves_q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_00921_gb300 import Plan
    from paper_1507_00921_gb300.fit import fit_adam
    link = synth.link(40)
    waves = []
    for k in range(3):
        tx, sym, bits = synth.pm_qpsk_waveform(2 ** 13, synth.BASE_SEED + 900 + k, 2.0)
        r = olink.forward(tx, link, FS, steps_per_span=20, ase_seed=synth.BASE_SEED + 950 + k)
        waves.append((r.astype(np.complex64), sym, bits))
    n = waves[0][0].shape[-1]
    nc = 16
    c0 = np.full(nc + 1, 1.0 / (2 * nc + 1), dtype=np.float32)
    x = torch.from_numpy(np.stack([w[0] for w in waves[:2]])).cuda()
    s = torch.from_numpy(np.stack([w[1] for w in waves[:2]]).astype(np.complex64)).cuda()
    with Plan(link, FS, n, n_waveforms=2, method="essfm", n_steps=1, n_taps=nc, fft_size=4096) as plan:
        c, losses = fit_adam(plan, x, s, coeffs0=c0, n_iter=200, lr=1e-2)
    assert losses[-1] < 0.9 * losses[0], (losses[0], losses[-1])
    r, sym, bits = waves[2]
    qs = {}
    for name, coeffs in (("start", c0), ("fitted", c)):
        with Plan(link, FS, n, method="essfm", n_steps=1, n_taps=nc, coeffs=coeffs, fft_size=4096) as plan:
            out = plan.run(torch.from_numpy(r[None]).cuda()).cpu().numpy()[0]
        qs[name] = rx.evaluate(out.astype(np.complex128), sym, bits)["q_db"]
    print(f"\nloss {losses[0]:.4f} -> {losses[-1]:.4f}; test Q start {qs['start']:.2f} dB, fitted {qs['fitted']:.2f} dB")
    assert qs["fitted"] > qs["start"] + 0.1
