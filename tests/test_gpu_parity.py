"""Parity of the CUDA DBP path (through the C ABI) with the FP64 oracle, element by
element.  Tolerance (FP32 path): relative RMS error over all outputs <= 1e-5 and every
sample within 1e-4 of the reference RMS amplitude."""
import numpy as np
import pytest

import synth
from oracle import dbp as odbp
from oracle import fiber

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


def gpu_dbp(torch, x, link, **kw):
    from paper_1507_00921_gb300 import Plan
    nw, _, n = x.shape
    with Plan(link, FS, n, n_waveforms=nw, **kw) as plan:
        xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = plan.run(xd)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.complex128), plan.info


def oracle_cfg(link, kw, info):
    nc = kw.get("n_taps", 0)
    essfm = kw.get("method", "essfm") == "essfm"
    coeffs = kw.get("coeffs")
    if coeffs is not None:
        coeffs = np.asarray(coeffs, dtype=np.float32).astype(np.float64)
        coeffs = coeffs.reshape(kw["n_steps"], nc + 1) if kw.get("coeffs_per_step") else coeffs
    return fiber.make_config(link, FS, kw.get("n_steps", 1), nc, kw["fft_size"], coeffs=coeffs,
                             overlap=info.overlap, boundary=kw.get("boundary", "periodic"), essfm=essfm,
                             step_len_m=kw.get("step_len_m"), gamma_eff=kw.get("gamma_eff"))


def compare(got, ref):
    err = got - ref
    rms_ref = np.sqrt(np.mean(np.abs(ref) ** 2))
    rel_rms = np.sqrt(np.mean(np.abs(err) ** 2)) / rms_ref
    max_rel = np.max(np.abs(err)) / rms_ref
    return rel_rms, max_rel


CASES = [
    # id, spans, n, n_wave, dBm, plan kwargs
    ("cfg1_essfm1_nc8_N1024", 10, 2 ** 15, 1, 2.0, dict(method="essfm", n_steps=1, n_taps=8, fft_size=1024)),
    ("cfg1_ssfm20_N1024", 10, 2 ** 15, 1, 2.0, dict(method="ssfm", n_steps=20, n_taps=0, fft_size=1024)),
    ("3200km_essfm1_nc32_N4096_ragged", 40, 2 ** 14 + 123, 2, 2.0,
     dict(method="essfm", n_steps=1, n_taps=32, fft_size=4096)),
    ("3200km_essfm2_nc16_N4096_zero", 40, 3 * 2600 + 7, 1, 4.0,
     dict(method="essfm", n_steps=2, n_taps=16, fft_size=4096, boundary="zero")),
    ("3200km_essfm4_nc32_N8192", 40, 2 ** 15, 1, 2.0, dict(method="essfm", n_steps=4, n_taps=32, fft_size=8192)),
    # unequal steps: one H table per step (the N = 8192 ESSFM kernel that keeps H in
    # shared memory; equal steps keep one H in tensor memory)
    ("3200km_essfm3_nc16_N8192_unequal_steps", 40, 2 ** 15 + 77, 2, 2.0,
     dict(method="essfm", n_steps=3, n_taps=16, fft_size=8192, step_len_m=np.array([1.4e6, 1.0e6, 0.8e6]))),
    ("3200km_ssfm1_N8192_zero", 40, 20000, 2, 6.0, dict(method="ssfm", n_steps=1, fft_size=8192, boundary="zero")),
    ("3200km_ssfm5_N2048", 40, 5000, 3, 0.0, dict(method="ssfm", n_steps=5, fft_size=2048)),
    ("3200km_ssfm20_N4096", 40, 2 ** 14, 1, 2.0, dict(method="ssfm", n_steps=20, fft_size=4096)),
    ("160km_essfm1_nc1_N512", 2, 3001, 2, 2.0, dict(method="essfm", n_steps=1, n_taps=1, fft_size=512)),
    ("800km_essfm3_nc4_N512", 10, 4000, 1, 2.0, dict(method="essfm", n_steps=3, n_taps=4, fft_size=512,
                                                    overlap=416)),
    ("800km_essfm1_nc8_N2048_tiny_n", 10, 100, 1, 2.0, dict(method="essfm", n_steps=1, n_taps=8, fft_size=2048)),
    ("800km_essfm1_nc8_N1024_one_sample", 10, 1, 1, 2.0, dict(method="essfm", n_steps=1, n_taps=8, fft_size=1024)),
    ("800km_essfm_nc0_N1024", 10, 5000, 1, 2.0, dict(method="essfm", n_steps=2, n_taps=0, fft_size=1024)),
    # largest filter (N_c = 64, every tap block) and largest step count (N_s = 1024)
    ("3200km_essfm1_nc64_N8192_max_taps", 40, 2 ** 14 + 9, 1, 2.0,
     dict(method="essfm", n_steps=1, n_taps=64, fft_size=8192)),
    ("160km_ssfm1024_N512_max_steps", 2, 2000, 1, 2.0, dict(method="ssfm", n_steps=1024, fft_size=512)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_with_oracle(torch_cuda, case):
    name, spans, n, nw, dbm, kw = case
    link = synth.link(spans)
    nc = kw.get("n_taps", 0)
    if kw.get("method") == "essfm" and nc > 0:
        c = 0.6 * np.exp(-np.arange(nc + 1) / max(1.0, nc / 3.0))
        kw = dict(kw, coeffs=(c / (c[0] + 2 * c[1:].sum())).astype(np.float32))
    x = synth.random_field(nw, n, synth.dbm_to_w(dbm), seed=1000 + len(name))
    got, info = gpu_dbp(torch_cuda, x, link, **kw)
    cfg = oracle_cfg(link, kw, info)
    ref = odbp.dbp(x.astype(np.complex64).astype(np.complex128), cfg)
    rel_rms, max_rel = compare(got, ref)
    # Every step applies the same FP32-rounded twiddle factors and dispersion table, so
    # their errors add coherently from step to step (about 8.3e-8 per step measured);
    # beyond ~100 steps the bound 1e-7 N_s takes over from 1e-5.
    ns = kw.get("n_steps", 1)
    tol_rms, tol_max = max(TOL_RMS, 1e-7 * ns), max(TOL_MAX, 4e-7 * ns)
    print(f"\n{name}: relative RMS error {rel_rms:.3e}, max error / RMS {max_rel:.3e}")
    assert rel_rms <= tol_rms, (rel_rms, max_rel)
    assert max_rel <= tol_max, (rel_rms, max_rel)


def test_per_step_coefficients_and_nonuniform_steps(torch_cuda):
    link = synth.link(40)
    dz = np.array([0.5e6, 1.2e6, 1.5e6])
    c = np.array([[0.5, 0.2, 0.05, 0.01, 0.0],
                  [0.3, 0.2, 0.1, 0.05, 0.02],
                  [0.6, 0.1, 0.05, 0.0, -0.01]], dtype=np.float32)
    kw = dict(method="essfm", n_steps=3, n_taps=4, coeffs=c.ravel(), coeffs_per_step=True, step_len_m=dz,
              fft_size=4096)
    x = synth.random_field(2, 12000, synth.dbm_to_w(3.0), seed=77)
    got, info = gpu_dbp(torch_cuda, x, link, **kw)
    cfg = oracle_cfg(link, kw, info)
    ref = odbp.dbp(x.astype(np.complex64).astype(np.complex128), cfg)
    rel_rms, max_rel = compare(got, ref)
    assert rel_rms <= TOL_RMS and max_rel <= TOL_MAX, (rel_rms, max_rel)


def test_set_coeffs_takes_effect(torch_cuda):
    from paper_1507_00921_gb300 import Plan
    torch = torch_cuda
    link = synth.link(10)
    x = synth.random_field(1, 8192, synth.dbm_to_w(2.0), seed=78).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    c1 = np.array([0.5, 0.2, 0.05], dtype=np.float32)
    c2 = np.array([0.9, 0.05, 0.0], dtype=np.float32)
    with Plan(link, FS, 8192, method="essfm", n_steps=1, n_taps=2, coeffs=c1, fft_size=1024) as plan:
        plan.set_coeffs(c2)
        got = plan.run(xd).cpu().numpy().astype(np.complex128)
        cfg = fiber.make_config(link, FS, 1, 2, 1024, coeffs=c2.astype(np.float64), overlap=plan.info.overlap)
    ref = odbp.dbp(x.astype(np.complex128), cfg)
    rel_rms, max_rel = compare(got, ref)
    assert rel_rms <= TOL_RMS and max_rel <= TOL_MAX


def test_run_host_matches_device_path(torch_cuda):
    from paper_1507_00921_gb300 import Plan
    torch = torch_cuda
    link = synth.link(40)
    x = synth.random_field(9, 6000, synth.dbm_to_w(2.0), seed=79).astype(np.complex64)
    with Plan(link, FS, 6000, n_waveforms=9, method="essfm", n_steps=1, n_taps=8, fft_size=4096) as plan:
        dev = plan.run(torch.from_numpy(x).cuda()).cpu().numpy()
        host = plan.run_host(torch.from_numpy(x).pin_memory()).numpy()
        host2 = plan.run_host(torch.from_numpy(x)).numpy()
    assert np.array_equal(dev, host)
    assert np.array_equal(dev, host2)


def test_alias_rejected(torch_cuda):
    from paper_1507_00921_gb300 import Plan, DBPError
    torch = torch_cuda
    link = synth.link(10)
    with Plan(link, FS, 4096, method="ssfm", n_steps=1, fft_size=1024) as plan:
        x = torch.zeros(1, 2, 4096, dtype=torch.complex64, device="cuda")
        with pytest.raises(DBPError) as e:
            plan.run(x, out=x)
        assert e.value.code == -6


@pytest.mark.parametrize("method,ns,nc,fft,nw", [("essfm", 1, 32, 4096, 8), ("essfm", 1, 32, 8192, 8),
                                                 ("ssfm", 20, 0, 4096, 8), ("essfm", 1, 32, 8192, 128),
                                                 ("essfm", 2, 32, 8192, 128)])
def test_full_size_3200km_sampled_blocks(torch_cuda, method, ns, nc, fft, nw):
    """Full 3200 km workload (2 x 524288 samples per waveform; batches of 8, and of 128
    as the benchmark launches it) in the benchmark's launch configuration; sampled
    blocks of the first, a middle and the last waveform checked against the oracle."""
    from paper_1507_00921_gb300 import Plan
    torch = torch_cuda
    link = synth.link(40)
    n = 2 * 2 ** 18
    x = synth.received_like(nw, 2 ** 18, 2.0, seed=4242, distinct=4)
    coeffs = None
    if nc:
        c = 0.6 * np.exp(-np.arange(nc + 1) / 10.0)
        coeffs = (c / (c[0] + 2 * c[1:].sum())).astype(np.float32)
    kw = dict(method=method, n_steps=ns, n_taps=nc, fft_size=fft, coeffs=coeffs)
    with Plan(link, FS, n, n_waveforms=nw, **kw) as plan:
        out = plan.run(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        info = plan.info
    cfg = oracle_cfg(link, kw, info)
    rng = np.random.default_rng(5)
    v = info.valid
    for w in sorted({0, 5 * nw // 8 + 2, nw - 1}):
        ids = np.unique(np.concatenate([[0, info.n_blocks - 1], rng.integers(0, info.n_blocks, 6)]))
        ref = odbp.dbp_blocks(x[w].astype(np.complex128), cfg, ids)         # [k, 2, V]
        for j, b in enumerate(ids):
            lo, hi = b * v, min((b + 1) * v, n)
            rel_rms, max_rel = compare(got[w][:, lo:hi].astype(np.complex128), ref[j][:, : hi - lo])
            assert rel_rms <= TOL_RMS and max_rel <= TOL_MAX, (w, b, rel_rms, max_rel)


SCHEME_CASES = [
    # id, spans, n, nw, kw  (per-step scheme: one pass per step; FFE: linear sub-step only)
    ("ffe_3200km_N4096", 40, 2 ** 14 + 5, 2, dict(method="ffe", n_steps=1, fft_size=4096)),
    ("ffe_800km_N1024_zero", 10, 5000, 1, dict(method="ffe", n_steps=1, fft_size=1024, boundary="zero")),
    ("perstep_ssfm20_3200km_N512", 40, 6000, 1, dict(method="ssfm", n_steps=20, fft_size=512, scheme="per_step")),
    ("perstep_ssfm20_3200km_N1024", 40, 2 ** 14, 2, dict(method="ssfm", n_steps=20, fft_size=1024,
                                                          scheme="per_step")),
    ("perstep_essfm4_nc16_3200km_N1024", 40, 9000, 1, dict(method="essfm", n_steps=4, n_taps=16, fft_size=1024,
                                                           scheme="per_step")),
    ("perstep_essfm3_nc8_nonuniform_N2048_zero", 40, 7000, 1,
     dict(method="essfm", n_steps=3, n_taps=8, fft_size=2048, scheme="per_step", boundary="zero",
          step_len_m=np.array([1.0e6, 1.5e6, 0.7e6]))),
]


@pytest.mark.parametrize("case", SCHEME_CASES, ids=[c[0] for c in SCHEME_CASES])
def test_ffe_and_per_step_scheme(torch_cuda, case):
    name, spans, n, nw, kw = case
    link = synth.link(spans)
    nc = kw.get("n_taps", 0)
    if nc:
        c = 0.6 * np.exp(-np.arange(nc + 1) / max(1.0, nc / 3.0))
        kw = dict(kw, coeffs=(c / (c[0] + 2 * c[1:].sum())).astype(np.float32))
    x = synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=2000 + len(name))
    got, info = gpu_dbp(torch_cuda, x, link, **kw)
    xr = x.astype(np.complex64).astype(np.complex128)
    coeffs = None if kw.get("coeffs") is None else np.asarray(kw["coeffs"], dtype=np.float32).astype(np.float64)
    if kw.get("scheme") == "per_step":
        cfgs = fiber.per_step_configs(link, FS, kw["n_steps"], nc, kw["fft_size"], coeffs=coeffs,
                                      boundary=kw.get("boundary", "periodic"), essfm=kw["method"] == "essfm",
                                      step_len_m=kw.get("step_len_m"))
        assert info.overlap == max(c.overlap for c in cfgs)
        ref = odbp.dbp_per_step(xr, cfgs)
    else:
        cfg = fiber.make_config(link, FS, kw["n_steps"], 0, kw["fft_size"], overlap=info.overlap,
                                boundary=kw.get("boundary", "periodic"), essfm=False,
                                gamma_eff=np.zeros(kw["n_steps"]))
        ref = odbp.dbp(xr, cfg)
    rel_rms, max_rel = compare(got, ref)
    print(f"\n{name}: relative RMS error {rel_rms:.3e}, max error / RMS {max_rel:.3e}")
    assert rel_rms <= TOL_RMS and max_rel <= TOL_MAX, (rel_rms, max_rel)


@pytest.mark.parametrize("n_pols", [2, 1])
def test_unaligned_buffers_match_aligned(torch_cuda, n_pols):
    """Input and output buffers that start 8 bytes past a 16-byte boundary (a view one
    complex sample into a larger allocation): the kernel's bulk output copies need 16-byte
    alignment, so it must take the per-thread store path, and its bulk L2 prefetch trims
    the window inward; the results must equal those of aligned buffers bit for bit."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    link = synth.link(40, manakov_factor=1.0 if n_pols == 1 else 8.0 / 9.0)
    n, nw = 2 ** 15, 2
    shape = (nw, n_pols, n) if n_pols == 2 else (nw, n)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.BASE_SEED + 1300)
    x = (torch.randn(shape, dtype=torch.complex64, device="cuda", generator=gen) * 0.03).contiguous()
    numel = x.numel()
    xbuf = torch.zeros(numel + 1, dtype=torch.complex64, device="cuda")
    ybuf = torch.zeros(numel + 1, dtype=torch.complex64, device="cuda")
    xu = xbuf[1:].view(shape)
    yu = ybuf[1:].view(shape)
    xu.copy_(x)
    assert xu.data_ptr() % 16 == 8 and yu.data_ptr() % 16 == 8
    with Plan(link, FS, n, n_waveforms=nw, n_pols=n_pols, method="essfm", n_steps=1, n_taps=32,
              fft_size=8192) as plan:
        ya = plan.run(x)
        plan.run(xu, yu)
        torch.cuda.synchronize()
    assert torch.equal(ya, yu)
    assert ybuf[0].item() == 0


def test_block_length_chosen_by_the_planner(torch_cuda):
    """fft_size = 0 (the Section III operation-count optimum chosen by the planner) runs the
    chosen block length and matches the oracle at that geometry."""
    from paper_1507_00921_gb300 import Plan
    torch = torch_cuda
    link = synth.link(20)
    n = 30000
    c = 0.6 * np.exp(-np.arange(17) / 5.0)
    kw = dict(method="essfm", n_steps=2, n_taps=16, coeffs=(c / (c[0] + 2 * c[1:].sum())).astype(np.float32))
    x = synth.random_field(2, n, synth.dbm_to_w(2.0), seed=321)
    with Plan(link, FS, n, n_waveforms=2, fft_size=0, **kw) as plan:
        got = plan.run(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
        info = plan.info
    assert info.fft_size in (2048, 4096, 8192) and info.overlap < info.fft_size
    cfg = oracle_cfg(link, dict(kw, fft_size=info.fft_size), info)
    rel_rms, max_rel = compare(got, odbp.dbp(x, cfg))
    assert rel_rms <= TOL_RMS and max_rel <= TOL_MAX, (rel_rms, max_rel)
