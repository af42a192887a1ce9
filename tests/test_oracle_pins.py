"""Pins of the FP64 oracle against facts other than itself: textbook special cases,
closed forms, library routines, invariants of Eqs. 1-3, brute force, exact inverses.
CPU only."""
import math

import numpy as np
import pytest

import synth
from oracle import adjoint, dbp, dft, fiber, fit, link as olink, rx

FS = synth.SAMPLE_RATE


def crandn(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- (e) DFT / FFT
def test_naive_dft_textbook_cases():
    n = 64
    delta = np.zeros(n, complex)
    delta[0] = 1
    assert np.allclose(dft.naive_dft(delta), np.ones(n), atol=1e-15)
    m = 5
    tone = np.exp(2j * np.pi * m * np.arange(n) / n)
    want = np.zeros(n, complex)
    want[m] = n
    assert np.max(np.abs(dft.naive_dft(tone) - want)) < 1e-12
    # shift theorem: x[n-1] <-> X_k exp(-j 2 pi k / N)
    x = crandn(n, 1)
    lhs = dft.naive_dft(np.roll(x, 1))
    rhs = dft.naive_dft(x) * np.exp(-2j * np.pi * np.arange(n) / n)
    assert rel(lhs, rhs) < 1e-13


def test_fft_equals_brute_force_dft_64():
    x = crandn((4, 64), 2)
    assert rel(dft.fft(x), dft.naive_dft(x)) < 1e-13
    assert rel(dft.ifft(x), dft.naive_dft(x, inverse=True)) < 1e-13


@pytest.mark.parametrize("n", [2, 8, 256, 1024, 8192])
def test_fft_matches_library(n):
    x = crandn((2, n), n)
    assert rel(dft.fft(x), np.fft.fft(x)) < 1e-13
    assert rel(dft.ifft(dft.fft(x)), x) < 1e-14
    assert np.allclose(dft.fftfreq(n, FS), np.fft.fftfreq(n, 1 / FS), rtol=0, atol=1e-3)


# ---------------------------------------------------------------- (a) invariants
def test_linear_substep_is_unitary():
    x = crandn((3, 2, 1024), 3)
    y = dbp.linear_substep(x, FS, -2.17e-26, 1.6e6)
    # Parseval per block and polarization; |H| = 1
    assert np.allclose(np.sum(abs(y) ** 2, -1), np.sum(abs(x) ** 2, -1), rtol=1e-12)
    h = dbp.dispersion_tf(1024, FS, -2.17e-26, 3.2e6)
    assert np.max(np.abs(np.abs(h) - 1)) < 1e-15
    # two steps compose into one (H_a H_b = H_{a+b})
    y2 = dbp.linear_substep(dbp.linear_substep(x, FS, -2.17e-26, 0.7e6), FS, -2.17e-26, 0.9e6)
    assert rel(y2, dbp.linear_substep(x, FS, -2.17e-26, 1.6e6)) < 1e-11


def test_nonlinear_substeps_are_phase_only():
    y = crandn((2, 2, 512), 4)
    z = dbp.nl_substep_essfm(y, 0.8, np.array([0.5, 0.2, 0.1, 0.05]))
    assert np.max(np.abs(np.abs(z) - np.abs(y)) / np.abs(y)) < 1e-14
    z2 = dbp.nl_substep_ssfm(y, 0.8)
    assert np.max(np.abs(np.abs(z2) - np.abs(y)) / np.abs(y)) < 1e-14
    # both polarizations receive the same phase rotation (Manakov, Section II)
    ph = np.angle(z / y)
    assert np.max(np.abs(np.angle(np.exp(1j * (ph[..., 0, :] - ph[..., 1, :]))))) < 1e-12


def test_essfm_phase_brute_force():
    p = np.random.default_rng(5).random(37)
    c = np.array([0.7, 0.3, -0.2, 0.1])
    th = dbp.essfm_phase(p, 2.0, c)
    n = len(p)
    for k in range(n):
        want = c[0] * p[k] + sum(c[i] * (p[(k - i) % n] + p[(k + i) % n]) for i in range(1, 4))
        assert abs(th[k] - 2.0 * want) < 1e-14


# ---------------------------------------------------------------- (d) ESSFM C=[1] == SSFM
def test_essfm_unit_filter_equals_ssfm_bitwise():
    link = synth.link(10)
    r = crandn((2, 4096), 6) * 0.04
    a = fiber.make_config(link, FS, 3, 0, 1024, essfm=False)
    b = fiber.make_config(link, FS, 3, 0, 1024, essfm=True)
    c = fiber.make_config(link, FS, 3, 2, 1024, essfm=True, coeffs=[1.0, 0.0, 0.0],
                          overlap=a.overlap)
    za, zb, zc = dbp.dbp(r, a), dbp.dbp(r, b), dbp.dbp(r, c)
    assert np.array_equal(za, zb)
    assert np.array_equal(za, zc)


# ---------------------------------------------------------------- (c) Gaussian pulse
def test_gaussian_pulse_dispersion_closed_form():
    fs, n, t0 = 200e9, 4096, 50e-12
    beta2, z = -21.68e-27, 500e3
    t = (np.arange(n) - n // 2) / fs
    a0 = np.exp(-t ** 2 / (2 * t0 ** 2))
    got = dbp.linear_substep(a0, fs, beta2, z, backward=False)     # forward Eq. 1
    q = t0 ** 2 + 1j * beta2 * z
    want = t0 / np.sqrt(q) * np.exp(-t ** 2 / (2 * q))
    assert np.max(np.abs(got - want)) < 1e-12
    # backpropagation (inverse of Eq. 1) undoes it
    back = dbp.linear_substep(want, fs, beta2, z, backward=True)
    assert np.max(np.abs(back - a0)) < 1e-12


# ---------------------------------------------------------------- (b) gamma = 0
@pytest.mark.parametrize("n_steps", [1, 3, 8])
def test_gamma_zero_dbp_is_analytic_cd_compensation(n_steps):
    link = synth.link(4)
    tx, _, _ = synth.pm_qpsk_waveform(2 ** 11, 7, 0.0)
    rx_ = olink.forward(tx, link, FS, steps_per_span=4, gamma_scale=0.0)
    n = tx.shape[-1]
    cfg = fiber.make_config(link, FS, n_steps, 0, n, overlap=0, gamma_eff=np.zeros(n_steps))
    out = dbp.dbp(rx_, cfg)
    assert rel(out, tx) < 1e-12
    # and equals one analytic CD compensation exp(+j beta2 w^2 L / 2)
    L = link["n_spans"] * link["span_len_m"]
    cd = dbp.linear_substep(rx_, FS, cfg.beta2, L, backward=True)
    assert rel(out, cd) < 1e-12


def test_overlap_save_converges_to_full_length():
    link = synth.link(10)
    tx, _, _ = synth.pm_qpsk_waveform(2 ** 12, 8, 0.0)
    rx_ = olink.forward(tx, link, FS, steps_per_span=2, gamma_scale=0.0)
    errs = []
    for o in [96, 200, 344, 600]:
        cfg = fiber.make_config(link, FS, 1, 0, 2048, overlap=o, gamma_eff=[0.0])
        errs.append(rel(dbp.dbp(rx_, cfg), tx))
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3


# ---------------------------------------------------------------- (f) link + DBP
def test_link_exact_inverse_recovers_tx():
    link = synth.link(3)
    tx, _, _ = synth.pm_qpsk_waveform(2 ** 11, 9, 3.0)
    r = olink.forward(tx, link, FS, steps_per_span=20)
    assert rel(r, tx) > 0.5                      # the channel really distorts
    back = olink.inverse(r, link, FS, steps_per_span=20)
    assert rel(back, tx) < 1e-11


def test_substep_effective_length_quadrature_and_limit():
    """The forward simulator's nonlinear weight of a sub-step of length h is the integral
    over the sub-step of the power relative to its midpoint value (Strang splitting with
    the rotation at the midpoint), exp(alpha h/2)(1 - exp(-alpha h))/alpha: checked
    against numerical quadrature of exp(-alpha (z - h/2)) over [0, h], and its alpha -> 0
    limit h."""
    from scipy.integrate import quad
    alpha = fiber.alpha_per_m(0.2)
    for h in (80.0, 3.2e3, 8e3, 80e3):
        want, _ = quad(lambda z: math.exp(-alpha * (z - h / 2.0)), 0.0, h, epsabs=0, epsrel=1e-13)
        assert abs(olink._mid_heff(alpha, h) - want) <= 1e-12 * want
    assert olink._mid_heff(0.0, 8e3) == 8e3
    for a in (1e-9, 1e-12):
        assert abs(olink._mid_heff(a, 8e3) - 8e3) < 1e-6 * 8e3


def test_forward_cw_nonlinear_phase_is_gamma_p_leff():
    """Section II: a constant-envelope (CW) field is untouched by dispersion, so one span of
    the forward simulator rotates it by exactly -gamma m P_0 L_eff (L_eff = (1 - e^{-alpha
    L})/alpha) and the EDFA restores its amplitude, whatever the number of sub-steps.  A
    wrong sub-step weight (e.g. the midpoint factor left out) moves the phase by ~20 % at
    ten sub-steps per span."""
    link = synth.link(1)
    p0 = synth.dbm_to_w(4.0)
    cw = np.full((2, 256), math.sqrt(p0) + 0j)
    alpha = fiber.alpha_per_m(0.2)
    leff = (1.0 - math.exp(-alpha * 80e3)) / alpha
    gam = 1.3e-3 * 8.0 / 9.0
    want = -gam * 2 * p0 * leff                    # joint intensity of both polarizations
    for sps in (1, 10, 100):
        u = olink.forward(cw, link, FS, steps_per_span=sps)
        assert np.allclose(np.abs(u), math.sqrt(p0), rtol=1e-12)
        assert np.allclose(np.angle(u), want, rtol=0, atol=1e-12)


def test_ase_variance_closed_form():
    """Section IV link (80 km spans, 0.2 dB/km, EDFA gain 16 dB, noise figure 5 dB) at
    f_s = 56 GSa/s: n_sp h nu (G - 1) f_s with n_sp = F G / (2 (G - 1)) is F G h nu f_s / 2
    per sample per polarization per amplifier, 4.517e-7 W (h nu at 1550 nm = 1.2816e-19 J),
    so 4.5e-6 W after 10 spans and 1.8e-5 W after 40."""
    link = synth.link(10)
    var = olink.ase_variance(link, FS)
    g = 10.0 ** 1.6                                 # 80 km x 0.2 dB/km = 16 dB
    f = 10.0 ** 0.5
    hnu = 6.62607015e-34 * 299792458.0 / 1550e-9
    assert abs(hnu - 1.2816e-19) < 1e-23
    assert abs(var - f * g * hnu * FS / 2.0) <= 1e-12 * var
    assert abs(var - 4.517e-7) < 1e-9
    assert abs(10 * var - 4.5e-6) < 0.05e-6
    assert abs(40 * var - 1.8e-5) < 0.05e-5


@pytest.mark.parametrize("n_spans,snr_db", [(10, 28.5), (40, 22.4)])
def test_forward_ase_accumulates_to_closed_form(n_spans, snr_db):
    """A zero signal through the forward simulator collects one amplifier's ASE per span
    (the span loss and the EDFA gain cancel for the noise already present): mean power per
    sample per polarization n_spans x 4.517e-7 W.  In the 28 GHz band of the 28 GBaud
    signal (half of the 56 GHz sampled band) that is an SNR of 28.5 dB after 10 spans and
    22.4 dB after 40 at 2 dBm per polarization."""
    link = synth.link(n_spans)
    n = 2 ** 16
    u = olink.forward(np.zeros((2, n), complex), link, FS, steps_per_span=1, ase_seed=7 + n_spans)
    p = np.mean(np.abs(u) ** 2)
    want = n_spans * 4.517e-7
    assert abs(p - want) < 0.015 * want            # 2^17 exponential samples: 0.28 % std
    spec = np.abs(np.fft.fft(u, axis=-1)) ** 2 / n
    f = np.fft.fftfreq(n, 1.0 / FS)
    inband = np.sum(spec[:, np.abs(f) < 14e9]) / (2 * n)   # per sample per polarization
    snr = 10.0 * math.log10(synth.dbm_to_w(2.0) / inband)
    assert abs(snr - snr_db) < 0.1, snr



def test_single_polarization_scalar_case():
    """One polarization (the scalar form Eq. 3 extends, P_k = |y_k|^2): (i) a CW field is
    untouched by dispersion (H(0) = 1), so every step rotates it by gamma_eff_s (c_0 +
    2 sum_i c_i) |A|^2 -- closed form for the whole DBP; (ii) on [1, n] the oracle equals
    the dual-polarization oracle with the second polarization zero; (iii) the scalar link
    (manakov factor 1) is inverted exactly."""
    link = synth.link(4, manakov_factor=1.0)
    n, amp = 4096, 0.07
    cw = np.full((1, n), amp * np.exp(0.3j))
    c = np.array([0.5, 0.2, 0.05, 0.01])
    cfg = fiber.make_config(link, FS, 3, 3, 1024, coeffs=c)
    phase = np.sum(cfg.gamma_eff) * (c[0] + 2 * c[1:].sum()) * amp ** 2
    np.testing.assert_allclose(dbp.dbp(cw, cfg), cw * np.exp(1j * phase), rtol=0, atol=1e-12)

    tx, _, _ = synth.pm_qpsk_waveform(2 ** 11, 31, 2.0)
    r1 = olink.forward(tx[:1], link, FS, steps_per_span=20)
    r2 = np.concatenate([r1, np.zeros_like(r1)], axis=0)
    for method_cfg in (fiber.make_config(link, FS, 1, 8, 1024), fiber.make_config(link, FS, 5, 0, 1024)):
        z1 = dbp.dbp(r1, method_cfg)
        z2 = dbp.dbp(r2, method_cfg)
        np.testing.assert_array_equal(z1[0], z2[0])
        assert not np.any(z2[1])
    assert rel(r1, tx[:1]) > 0.5
    assert rel(olink.inverse(r1, link, FS, steps_per_span=20), tx[:1]) < 1e-11

def test_ssfm_dbp_error_falls_with_steps():
    link = synth.link(10)
    tx, _, _ = synth.pm_qpsk_waveform(2 ** 11, 10, 2.0)
    r = olink.forward(tx, link, FS, steps_per_span=20)
    n = tx.shape[-1]
    errs = []
    for ns in [1, 2, 5, 10, 20, 40]:
        cfg = fiber.make_config(link, FS, ns, 0, n, overlap=0)
        errs.append(rel(dbp.dbp(r, cfg), tx))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.2 * errs[0]


@pytest.mark.slow
def test_dbp_beats_ffe_with_ase():
    link = synth.link(40)
    tx, sym, bits = synth.pm_qpsk_waveform(2 ** 12, 11, 2.0)
    r = olink.forward(tx, link, FS, steps_per_span=10, ase_seed=12)
    n = tx.shape[-1]
    ffe = fiber.make_config(link, FS, 1, 0, n, overlap=0, gamma_eff=[0.0])
    ss40 = fiber.make_config(link, FS, 40, 0, n, overlap=0)
    q_ffe = rx.evaluate(dbp.dbp(r, ffe), sym, bits)["q_db"]
    q_40 = rx.evaluate(dbp.dbp(r, ss40), sym, bits)["q_db"]
    assert q_40 > q_ffe + 1.0


# ---------------------------------------------------------------- receiver
def test_receiver_noise_free_and_awgn():
    tx, sym, bits = synth.pm_qpsk_waveform(2 ** 14, 13, 0.0)
    e = rx.evaluate(tx, sym, bits)
    assert e["bit_errors"] == 0 and e["snr_eff"] > 1e10
    # white noise at a known in-band SNR: SNR_eff and BER follow the QPSK closed form
    p = synth.dbm_to_w(0.0)
    snr = 10 ** (8.0 / 10)
    noisy = tx + synth.awgn(tx.shape, p / snr * 2, 14)      # per-sample var at 2 sps
    e = rx.evaluate(noisy, sym, bits)
    assert abs(e["q_db"] - 8.0) < 0.15
    ber = 0.5 * math.erfc(math.sqrt(snr / 2))
    assert abs(e["ber"] - ber) < 0.15 * ber


# ---------------------------------------------------------------- steps / memory
def test_step_effective_lengths():
    link = synth.link(40)
    alpha = fiber.alpha_per_m(0.2)
    leff = (1 - math.exp(-alpha * 80e3)) / alpha                # Section II, Eq. 2 note
    assert abs(leff - 21.169e3) < 2.0
    g = 1.3e-3 * 8 / 9
    dz, geff = fiber.step_table(link, 40)                      # one span per step
    assert np.allclose(geff, g * leff, rtol=1e-13)
    dz, geff = fiber.step_table(link, 20)                      # two spans per step
    assert np.allclose(geff, 2 * g * leff, rtol=1e-13)
    for ns in [1, 3, 7, 16]:                                   # total is invariant
        dz, geff = fiber.step_table(link, ns)
        assert abs(np.sum(geff) - 40 * g * leff) < 1e-9 * 40 * g * leff
        assert abs(np.sum(dz) - 3.2e6) < 1e-6


def test_memory_and_dispersion_against_paper_values():
    # SMF with D = 17 ps/(nm km) at 1550 nm: beta2 ~ -21.7 ps^2/km (the paper uses 21)
    b2 = fiber.beta2_from_D(17.0, 1550e-9)
    assert abs(b2 * 1e27 + 21.7) < 0.05
    # Section III: 50 GHz over about 3000 km of SMF gives M ~ 1024 samples
    m = fiber.channel_memory(21e-27, 3000e3, 50e9)
    assert abs(m - 1024) / 1024 < 0.04
    assert fiber.overlap_rule(1367.15, 1, 32) == 1432


# ---------------------------------------------------------------- coefficient fit
def test_fit_recovers_known_coefficients():
    link = synth.link(10)
    r = crandn((2, 8192), 15) * 0.04
    c_true = np.array([0.4, 0.2, 0.1, -0.05, 0.02])
    cfg = fiber.make_config(link, FS, 1, 4, 1024, coeffs=c_true)
    target = dbp.dbp(r, cfg)
    got = fit.fit_single_step(r, target, cfg)
    assert np.max(np.abs(got - c_true)) < 1e-9


# ---------------------------------------------------------------- adjoint
def _adj_case(essfm=True, boundary="periodic"):
    link = synth.link(2)
    r = crandn((2, 640), 16) * 0.05
    n_c = 3 if essfm else 0
    c = np.array([[0.6, 0.2, 0.1, -0.05], [0.5, 0.25, -0.1, 0.05]])[:, : n_c + 1]
    cfg = fiber.make_config(link, FS, 2, n_c, 256, coeffs=c, overlap=96, boundary=boundary,
                            essfm=essfm)
    cfg.gamma_eff = np.array([250.0, 300.0])
    v = crandn((2, 640), 17)
    return r, cfg, v


def _loss(r, cfg, v):
    return float(np.real(np.sum(np.conj(v) * dbp.dbp(r, cfg))))


@pytest.mark.parametrize("boundary", ["periodic", "zero"])
def test_adjoint_matches_central_differences(boundary):
    r, cfg, v = _adj_case(boundary=boundary)
    g_in, g_c, g_g, g_dz = adjoint.dbp_vjp(r, cfg, v)

    def fd(setter, h):
        import copy
        a, b = copy.deepcopy(cfg), copy.deepcopy(cfg)
        ra, rb = r.copy(), r.copy()
        setter(a, ra, +h)
        setter(b, rb, -h)
        return (_loss(ra, a, v) - _loss(rb, b, v)) / (2 * h)

    def check(an, num):
        assert abs(an - num) <= 1e-5 * max(abs(num), 1e-3 * np.linalg.norm(g_c)), (an, num)

    for s in range(2):
        for i in range(4):
            def set_c(c, rr, h, s=s, i=i):
                c.coeffs[s, i] += h
            check(g_c[s, i], fd(set_c, 1e-4))

        def set_g(c, rr, h, s=s):
            c.gamma_eff[s] += h
        check(g_g[s], fd(set_g, 1e-4 * cfg.gamma_eff[s]))

        def set_dz(c, rr, h, s=s):
            c.dz[s] += h
        check(g_dz[s], fd(set_dz, 1e-4 * cfg.dz[s]))
    for p, k in [(0, 0), (1, 5), (0, 300), (1, 639)]:
        def set_re(c, rr, h, p=p, k=k):
            rr[p, k] += h

        def set_im(c, rr, h, p=p, k=k):
            rr[p, k] += 1j * h
        check(g_in[p, k].real, fd(set_re, 1e-4 * 0.05))
        check(g_in[p, k].imag, fd(set_im, 1e-4 * 0.05))


def test_linear_adjoint_dot_product():
    r, cfg, v = _adj_case()
    cfg.gamma_eff = np.zeros(2)
    ux = dbp.dbp(r, cfg)
    g_in, *_ = adjoint.dbp_vjp(r, cfg, v)
    lhs = np.vdot(v, ux)            # <v, U x>
    rhs = np.vdot(g_in, r)          # <U^H v, x>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ---------------------------------------------------------------- per-step-pass scheme
def test_per_step_scheme_full_length_equals_fused():
    link = synth.link(10)
    r = crandn((2, 2048), 41) * 0.04
    fused = fiber.make_config(link, FS, 4, 3, 2048, coeffs=[0.5, 0.2, 0.1, 0.05], overlap=0)
    cfgs = fiber.per_step_configs(link, FS, 4, 3, 2048, coeffs=[0.5, 0.2, 0.1, 0.05], overlap=0)
    for c in cfgs:
        c.overlap = 0
    assert np.array_equal(dbp.dbp_per_step(r, cfgs), dbp.dbp(r, fused))


def test_per_step_scheme_overlap_rule_and_convergence():
    link = synth.link(40)
    cfgs = fiber.per_step_configs(link, FS, 20, 0, 512)
    assert all(c.overlap == 72 for c in cfgs)            # ceil(1367.2 / 20) = 69 -> 72
    tx, _, _ = synth.pm_qpsk_waveform(2 ** 11, 42, 0.0)
    r = olink.forward(tx, link, FS, steps_per_span=1, gamma_scale=0.0)
    errs = []
    for o in (72, 160, 320):
        c = fiber.per_step_configs(link, FS, 20, 0, 1024, overlap=o, ffe=True)
        errs.append(rel(dbp.dbp_per_step(r, c), tx))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3
