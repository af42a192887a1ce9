"""The CUDA adjoint (dbp_grad through the C ABI) against the FP64 oracle's adjoint and
against central finite differences of the FP64 oracle (h = 1e-4), for the loss
L = Re sum conj(v) DBP(x).  Tolerance: 1e-3 relative per gradient component (floor at
1e-3 of the vector's norm); input gradient: relative RMS 1e-4."""
import copy

import numpy as np
import pytest

import synth
from oracle import adjoint as oadj
from oracle import dbp as odbp
from oracle import fiber

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE
TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def coeffs_for(nc, ns, per_step, seed=3):
    g = np.random.default_rng(seed)
    c = 0.6 * np.exp(-np.arange(nc + 1) / max(1.0, nc / 3.0))
    c = c / (c[0] + 2 * c[1:].sum())
    if per_step:
        c = np.stack([c * (1 + 0.1 * g.standard_normal(nc + 1)) for _ in range(ns)])
    return c.astype(np.float32)


def close(got, ref):
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    floor = 1e-3 * np.linalg.norm(ref)
    return np.all(np.abs(got - ref) <= TOL * np.maximum(np.abs(ref), floor)), np.max(
        np.abs(got - ref) / np.maximum(np.abs(ref), floor))


CASES = [
    # id, spans, n, nw, kw
    ("essfm1_nc16_N4096", 40, 9000, 2, dict(method="essfm", n_steps=1, n_taps=16, fft_size=4096)),
    ("essfm2_nc16_N4096_zero", 40, 7000, 1, dict(method="essfm", n_steps=2, n_taps=16, fft_size=4096,
                                                 boundary="zero")),
    ("essfm4_nc16_N4096_perstep", 40, 8000, 1, dict(method="essfm", n_steps=4, n_taps=16, fft_size=4096,
                                                    coeffs_per_step=True)),
    ("ssfm3_N2048", 10, 5000, 2, dict(method="ssfm", n_steps=3, fft_size=2048)),
    ("essfm3_nc8_N1024_nonuniform", 10, 4000, 1, dict(method="essfm", n_steps=3, n_taps=8, fft_size=1024,
                                                      step_len_m=np.array([2e5, 3.5e5, 2.5e5]))),
    ("essfm1_nc32_N8192", 40, 12000, 1, dict(method="essfm", n_steps=1, n_taps=32, fft_size=8192)),
    # N = 8192 keeps U and g in tensor memory across the steps of the reverse sweep
    ("essfm3_nc8_N8192_zero_perstep", 40, 17000, 1, dict(method="essfm", n_steps=3, n_taps=8, fft_size=8192,
                                                         boundary="zero", coeffs_per_step=True)),
    ("ssfm4_N8192", 40, 15000, 2, dict(method="ssfm", n_steps=4, fft_size=8192)),
    ("essfm2_nc4_N512_tiny_n", 2, 300, 1, dict(method="essfm", n_steps=2, n_taps=4, fft_size=512)),
]


def run_case(torch, spans, n, nw, kw):
    from paper_1507_00921_gb300 import Plan
    link = synth.link(spans)
    nc, ns = kw.get("n_taps", 0), kw["n_steps"]
    if nc:
        kw = dict(kw, coeffs=coeffs_for(nc, ns, kw.get("coeffs_per_step", False)).ravel())
    x = synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=n).astype(np.complex64)
    v = synth.random_field(nw, n, 1.0, seed=n + 1).astype(np.complex64)
    with Plan(link, FS, n, n_waveforms=nw, **kw) as plan:
        xd, vd = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        g_in, d_c, d_g, d_z = plan.grad(xd, vd)
        torch.cuda.synchronize()
        out = (g_in.cpu().numpy(), d_c.cpu().numpy(), d_g.cpu().numpy(), d_z.cpu().numpy())
        ov = plan.info.overlap
    c = kw.get("coeffs")
    if c is not None:
        c = np.asarray(c, dtype=np.float64)
        c = c.reshape(ns, nc + 1) if kw.get("coeffs_per_step") else c
    cfg = fiber.make_config(link, FS, ns, nc, kw["fft_size"], coeffs=c, overlap=ov,
                            boundary=kw.get("boundary", "periodic"), essfm=kw["method"] == "essfm",
                            step_len_m=kw.get("step_len_m"))
    return x, v, cfg, out, kw


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_oracle(torch_cuda, case):
    name, spans, n, nw, kw = case
    x, v, cfg, (g_in, d_c, d_g, d_z), kw = run_case(torch_cuda, spans, n, nw, kw)
    ref_in = np.zeros_like(x, dtype=np.complex128)
    ref_c = np.zeros_like(cfg.coeffs)
    ref_g = np.zeros(cfg.n_steps)
    ref_z = np.zeros(cfg.n_steps)
    for w in range(nw):
        gi, gc, gg, gz = oadj.dbp_vjp(x[w].astype(np.complex128), cfg, v[w].astype(np.complex128))
        ref_in[w] = gi
        ref_c += gc
        ref_g += gg
        ref_z += gz
    if not kw.get("coeffs_per_step"):
        ref_c = ref_c.sum(axis=0)
    rel_in = np.linalg.norm(g_in - ref_in) / np.linalg.norm(ref_in)
    ok_c, e_c = close(d_c, ref_c)
    ok_g, e_g = close(d_g, ref_g)
    ok_z, e_z = close(d_z, ref_z)
    print(f"\n{name}: g_in rel {rel_in:.2e}, d_c {e_c:.2e}, d_gamma {e_g:.2e}, d_dz {e_z:.2e}")
    assert rel_in <= 1e-4
    assert ok_c and ok_g and ok_z, (e_c, e_g, e_z)


def test_adjoint_matches_central_differences(torch_cuda):
    """GPU gradients vs central finite differences of the FP64 oracle, h = 1e-4."""
    name, spans, n, nw, kw = CASES[2]
    x, v, cfg, (g_in, d_c, d_g, d_z), kw = run_case(torch_cuda, spans, n, nw, kw)
    xx, vv = x[0].astype(np.complex128), v[0].astype(np.complex128)

    def loss(c):
        return float(np.real(np.sum(np.conj(vv) * odbp.dbp(xx, c))))

    def fd(mutate, h):
        a, b = copy.deepcopy(cfg), copy.deepcopy(cfg)
        mutate(a, h)
        mutate(b, -h)
        return (loss(a) - loss(b)) / (2 * h)

    checks = []
    for s, i in [(0, 0), (1, 3), (3, 16), (2, 1)]:
        def m(c, h, s=s, i=i):
            c.coeffs[s, i] += h
        checks.append((d_c[s, i], fd(m, 1e-4)))
    for s in range(cfg.n_steps):
        def mg(c, h, s=s):
            c.gamma_eff[s] += h
        checks.append((d_g[s], fd(mg, 1e-4 * cfg.gamma_eff[s])))

        def mz(c, h, s=s):
            c.dz[s] += h
        checks.append((d_z[s], fd(mz, 1e-4 * cfg.dz[s])))
    for got, want in checks:
        assert abs(got - want) <= TOL * max(abs(want), 1e-6), (got, want)


def test_autograd_module(torch_cuda):
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    from paper_1507_00921_gb300.dbp import DBP
    link = synth.link(40)
    n = 6000
    x = torch.from_numpy(synth.random_field(1, n, synth.dbm_to_w(2.0), seed=9).astype(np.complex64)).cuda()
    t = torch.from_numpy(synth.random_field(1, n, synth.dbm_to_w(2.0), seed=10).astype(np.complex64)).cuda()
    with Plan(link, FS, n, method="essfm", n_steps=1, n_taps=4, fft_size=4096) as plan:
        mod = DBP(plan, coeffs=np.array([0.5, 0.2, 0.1, 0.05, 0.02], dtype=np.float32))
        xr = x.clone().requires_grad_(True)
        loss = (mod(xr) - t).abs().pow(2).mean()
        loss.backward()
        g_c = mod.coeffs.grad.clone()
        g_x = xr.grad.clone()
        # same gradient directly from dbp_grad with g_out = dL/dout = 2 (out - t) / numel
        out = plan.run(x)
        _, d_c, _, _ = plan.grad(x, (2.0 / out.numel()) * (out - t))
    assert torch.allclose(g_c.cuda(), d_c, rtol=1e-5, atol=1e-9)
    assert g_x.shape == x.shape and torch.isfinite(torch.view_as_real(g_x)).all()


def test_autograd_over_coeffs_gamma_and_step_lengths(torch_cuda):
    """DBPFunction.apply(x, c, gamma_eff, dz, plan) (Eqs. 1-3 with all three parameter
    sets as tensors): the forward output equals a plan built with those parameters, and
    the four gradients of L = Re sum conj(v) DBP(x) equal the FP64 oracle's adjoint and,
    for gamma_eff and dz, central finite differences of the oracle (h = 1e-4 relative)."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    from paper_1507_00921_gb300.dbp import DBPFunction
    link = synth.link(40)
    n, nw, ns, nc = 7000, 1, 3, 8
    c = coeffs_for(nc, ns, True)
    dz = np.array([1.1e6, 0.9e6, 1.2e6])
    x = synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=71).astype(np.complex64)
    v = synth.random_field(nw, n, 1.0, seed=72).astype(np.complex64)
    kw = dict(method="essfm", n_steps=ns, n_taps=nc, fft_size=4096, coeffs_per_step=True)
    with Plan(link, FS, n, n_waveforms=nw, **kw) as plan:
        ge = plan.info.step_gamma_eff * np.array([0.9, 1.05, 1.2])
        xd = torch.from_numpy(x).cuda().requires_grad_(True)
        vd = torch.from_numpy(v).cuda()
        ct = torch.tensor(c, requires_grad=True)
        gt = torch.tensor(ge, requires_grad=True)
        zt = torch.tensor(dz, requires_grad=True)
        out = DBPFunction.apply(xd, ct, gt, zt, plan)
        loss = (torch.conj(vd) * out).real.sum()
        loss.backward()
        ov = plan.info.overlap
        with Plan(link, FS, n, n_waveforms=nw, coeffs=c.ravel(), step_len_m=dz, gamma_eff=ge, overlap=ov,
                  **kw) as direct:
            ref_out = direct.run(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        assert torch.equal(out.detach(), ref_out)
        g_x, g_c, g_g, g_z = xd.grad.cpu().numpy(), ct.grad.numpy(), gt.grad.numpy(), zt.grad.numpy()
    cfg = fiber.make_config(link, FS, ns, nc, 4096, coeffs=c.astype(np.float64), overlap=ov, step_len_m=dz,
                            gamma_eff=ge)
    xx, vv = x[0].astype(np.complex128), v[0].astype(np.complex128)
    r_x, r_c, r_g, r_z = oadj.dbp_vjp(xx, cfg, vv)
    assert np.linalg.norm(g_x[0] - r_x) / np.linalg.norm(r_x) <= 1e-4
    for got, ref in ((g_c, r_c), (g_g, r_g), (g_z, r_z)):
        ok, e = close(got, ref)
        assert ok, e

    def loss_of(cf):
        return float(np.real(np.sum(np.conj(vv) * odbp.dbp(xx, cf))))

    for s in range(ns):
        for attr, got in (("gamma_eff", g_g[s]), ("dz", g_z[s])):
            h = 1e-4 * getattr(cfg, attr)[s]
            a, b = copy.deepcopy(cfg), copy.deepcopy(cfg)
            getattr(a, attr)[s] += h
            getattr(b, attr)[s] -= h
            fd = (loss_of(a) - loss_of(b)) / (2 * h)
            assert abs(got - fd) <= TOL * max(abs(fd), 1e-6), (attr, s, got, fd)


def test_gradient_is_bitwise_reproducible(torch_cuda):
    """Every partial sum is reduced in an order fixed by the problem's shape (per-warp rows,
    segments of rows, then the segments in order) and the input gradient sums its covering
    blocks in block order, so two calls, on two streams, give the same bits.  The size
    (16 waveforms, N = 4096, eight warp rows per block) spans several reduction segments."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    n, nw = 1 << 17, 16
    x = torch.from_numpy(synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=21).astype(np.complex64)).cuda()
    v = torch.from_numpy(synth.random_field(nw, n, 1.0, seed=22).astype(np.complex64)).cuda()
    with Plan(synth.link(40), FS, n, n_waveforms=nw, method="essfm", n_steps=2, n_taps=16, fft_size=4096,
              coeffs=coeffs_for(16, 2, True).ravel(), coeffs_per_step=True) as plan:
        assert plan.info.n_blocks * nw * 8 > 4 * 1024      # more than four reduction segments
        first = plan.grad(x, v)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())          # the plan's scratch is shared by its calls
        with torch.cuda.stream(s):
            second = plan.grad(x, v, stream=s)
        s.synchronize()
        torch.cuda.synchronize()
    for a, b in zip(first, second):
        assert torch.equal(a, b)
    assert all(torch.isfinite(torch.view_as_real(t) if t.is_complex() else t).all() for t in first)


def test_parameter_gradients_without_the_input_gradient(torch_cuda):
    """grad_in = NULL skips the overlap-add gather, so the first reduction kernel follows the
    adjoint kernel directly; the parameter gradients must be the same bits as with it."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Plan
    n, nw = 20000, 2
    x = torch.from_numpy(synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=31).astype(np.complex64)).cuda()
    v = torch.from_numpy(synth.random_field(nw, n, 1.0, seed=32).astype(np.complex64)).cuda()
    for kw in (dict(method="essfm", n_steps=2, n_taps=16, fft_size=4096, coeffs=coeffs_for(16, 2, False)),
               dict(method="ssfm", n_steps=3, fft_size=8192)):
        with Plan(synth.link(40), FS, n, n_waveforms=nw, **kw) as plan:
            full = plan.grad(x, v)
            part = plan.grad(x, v, need_input=False)
            torch.cuda.synchronize()
        assert part[0] is None
        for a, b in zip(full[1:], part[1:]):
            assert torch.equal(a, b), kw
