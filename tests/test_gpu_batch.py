"""Batched uneven workloads through one CUDA-graph launch of persistent kernels: every
job's output matches the FP64 oracle on sampled blocks (jobs of 2^12-2^18 symbols, the
uneven-batch workload's range) and its own dbp_run; replays are identical; streaming jobs
wait for their publish flag with a bounded spin and a never-published job ends in
DBP_ERR_TIMEOUT without hanging."""
import time

import numpy as np
import pytest

import synth
from oracle import dbp as odbp
from oracle import fiber

pytestmark = pytest.mark.gpu
FS = synth.SAMPLE_RATE


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def fft_for(spans, method, ns, nc):
    """Smallest supported block length at least twice the overlap."""
    from paper_1507_00921_gb300 import describe
    for n in (1024, 2048, 4096, 8192):
        try:
            info = describe(synth.link(spans), FS, 4096, method=method, n_steps=ns, n_taps=nc, fft_size=n)
        except Exception:
            continue
        if n >= 2 * info.overlap:
            return n
    return 8192


def make_jobs(torch, n_jobs, seed, max_log2=13, min_log2=9, specs=None):
    """Plans, device inputs and zeroed outputs of a seeded uneven job list; `specs`
    (if a list) receives each job's (link, plan keyword arguments)."""
    from paper_1507_00921_gb300 import Plan
    plans, ins, outs = [], [], []
    for k, jb in enumerate(synth.batch_jobs(n_jobs, seed, min_log2, max_log2)):
        n = jb["n_symbols"] * synth.SPS
        nc = jb["n_taps"]
        coeffs = None
        if nc:
            c = 0.6 * np.exp(-np.arange(nc + 1) / 8.0)
            coeffs = (c / (c[0] + 2 * c[1:].sum())).astype(np.float32)
        nw = 1 + (k % 3)
        fft = fft_for(jb["n_spans"], jb["method"], jb["n_steps"], nc)
        kw = dict(method=jb["method"], n_steps=jb["n_steps"], n_taps=nc, coeffs=coeffs, fft_size=fft,
                  boundary="zero" if k % 4 == 3 else "periodic")
        plans.append(Plan(synth.link(jb["n_spans"]), FS, n, n_waveforms=nw, **kw))
        if specs is not None:
            specs.append((synth.link(jb["n_spans"]), kw))
        x = synth.random_field(nw, n, synth.dbm_to_w(jb["launch_dbm"]), seed=jb["seed"]).astype(np.complex64)
        ins.append(torch.from_numpy(x).cuda())
        outs.append(torch.zeros_like(ins[-1]))
    return plans, ins, outs


def test_batch_equals_individual_runs_and_replays(torch_cuda):
    torch = torch_cuda
    from paper_1507_00921_gb300 import Batch
    plans, ins, outs = make_jobs(torch, 14, 501)
    assert len({p.info.fft_size for p in plans}) >= 2
    refs = [p.run(x) for p, x in zip(plans, ins)]
    with Batch(plans, ins, outs) as batch:
        batch.run()
        assert batch.status() == 0
        first = [o.clone() for o in outs]
        for o in outs:
            o.zero_()
        batch.run()
        assert batch.status() == 0
    for o, f, r in zip(outs, first, refs):
        assert torch.equal(o, f)
        assert torch.equal(o, r)               # the same arithmetic as the job's own dbp_run
    for p in plans:
        p.close()


def test_batch_matches_oracle_on_long_uneven_jobs(torch_cuda):
    """The batch kernel (its own instantiation: per-item parameter loads, table twiddles)
    against the FP64 oracle, on jobs of 2^12 to 2^18 symbols per polarization: the first,
    the last and random blocks of the first and the last waveform of every job, at the
    FP32 parity bar (relative RMS <= 1e-5, every sample within 1e-4 of the RMS)."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Batch
    specs = []
    plans, ins, outs = make_jobs(torch, 10, 2025, max_log2=18, min_log2=12, specs=specs)
    assert max(x.shape[-1] for x in ins) > 2 ** 18.9 and min(x.shape[-1] for x in ins) < 2 ** 14
    with Batch(plans, ins, outs) as batch:
        batch.run()
        assert batch.status() == 0
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    worst = 0.0
    for p, x, y, (link, kw) in zip(plans, ins, outs, specs):
        info = p.info
        xs, ys = x.cpu().numpy(), y.cpu().numpy()
        c = kw["coeffs"]
        cfg = fiber.make_config(link, FS, kw["n_steps"], kw["n_taps"], kw["fft_size"],
                                coeffs=None if c is None else c.astype(np.float64), overlap=info.overlap,
                                boundary=kw["boundary"], essfm=kw["method"] == "essfm")
        n, v = xs.shape[-1], info.valid
        for w in sorted({0, xs.shape[0] - 1}):
            ids = np.unique(np.concatenate([[0, info.n_blocks - 1], rng.integers(0, info.n_blocks, 3)]))
            ref = odbp.dbp_blocks(xs[w].astype(np.complex128), cfg, ids)
            for j, b in enumerate(ids):
                lo, hi = b * v, min((b + 1) * v, n)
                got = ys[w][:, lo:hi].astype(np.complex128)
                want = ref[j][:, : hi - lo]
                rms = np.sqrt(np.mean(np.abs(want) ** 2))
                rel_rms = np.sqrt(np.mean(np.abs(got - want) ** 2)) / rms
                max_rel = np.max(np.abs(got - want)) / rms
                worst = max(worst, rel_rms)
                assert rel_rms <= 1e-5 and max_rel <= 1e-4, (kw, w, b, rel_rms, max_rel)
    print(f"\nbatch vs oracle: worst relative RMS {worst:.2e}")
    for p in plans:
        p.close()


def test_streaming_publish_and_bounded_timeout(torch_cuda):
    torch = torch_cuda
    from paper_1507_00921_gb300 import Batch, _lib
    plans, ins, outs = make_jobs(torch, 4, 777, max_log2=11)
    refs = [p.run(x) for p, x in zip(plans, ins)]
    side = torch.cuda.Stream()
    with Batch(plans, ins, outs, streaming=True, timeout_us=20000) as batch:
        batch.run()
        for j in range(4):
            batch.publish(j, stream=side)
        assert batch.status() == 0
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
        for o in outs:
            o.zero_()
        t0 = time.time()
        batch.run()
        for j in (0, 1, 3):                       # job 2 is never published
            batch.publish(j, stream=side)
        assert batch.status() == _lib.DBP_ERR_TIMEOUT
        assert time.time() - t0 < 30.0
        for j in (0, 1, 3):
            assert torch.equal(outs[j], refs[j])
        assert outs[2].abs().max().item() == 0.0
    for p in plans:
        p.close()


def test_run_batch_one_shot(torch_cuda):
    torch = torch_cuda
    import ctypes as C
    from paper_1507_00921_gb300 import _lib
    plans, ins, outs = make_jobs(torch, 3, 99, max_log2=11)
    lib = _lib.load()
    arr = C.c_void_p * 3
    rc = lib.dbp_run_batch(arr(*[p._h.value for p in plans]), arr(*[x.data_ptr() for x in ins]),
                           arr(*[y.data_ptr() for y in outs]), 3, None)
    assert rc == 0
    for p, x, y in zip(plans, ins, outs):
        r = p.run(x)
        torch.cuda.synchronize()
        assert torch.equal(y, r)
        p.close()


def test_tensor_memory_twiddles_match_table_twiddles(torch_cuda):
    """At N = 8192 the forward kernel reads each thread's pass-1 twiddles from tensor
    memory, where they were stored once per kernel; the batch kernel forms them from the
    shared-memory tables every pass.  Both take the same FP32 product, so for an SSFM
    plan (which differs in nothing else) the two outputs are bit for bit identical."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Batch, Plan
    n, nw = 20000, 2
    x = torch.from_numpy(synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=818).astype(np.complex64)).cuda()
    with Plan(synth.link(40), FS, n, n_waveforms=nw, method="ssfm", n_steps=2, fft_size=8192) as plan:
        y_run = plan.run(x)
        y_batch = torch.zeros_like(x)
        batch = Batch([plan], [x], [y_batch])
        batch.run()
        torch.cuda.synchronize()
        assert batch.status() == 0
        batch.close()
    assert torch.equal(y_run, y_batch)


def test_batch_every_block_length_against_runs_and_oracle(torch_cuda):
    """One batch with jobs at every block length (512 ... 8192), so that the persistent
    kernel runs units of 14, 7, 4, 2 and 1 blocks side by side: every job takes exactly the
    arithmetic of its own dbp_run (bitwise equal; ESSFM jobs of one or two steps take the
    hardware exponential in both), and sampled blocks of every job match the FP64
    oracle."""
    torch = torch_cuda
    from paper_1507_00921_gb300 import Batch, Plan
    specs = [  # spans, n, n_waveforms, plan keyword arguments
        (1, 3000, 2, dict(method="ssfm", n_steps=3, fft_size=512)),
        (1, 2501, 1, dict(method="essfm", n_steps=1, n_taps=8, fft_size=512, boundary="zero")),
        (4, 9000, 2, dict(method="ssfm", n_steps=5, fft_size=1024, boundary="zero")),
        (4, 7777, 3, dict(method="essfm", n_steps=3, n_taps=4, fft_size=1024)),
        (10, 20000, 1, dict(method="essfm", n_steps=2, n_taps=16, fft_size=2048)),
        (10, 12345, 2, dict(method="ssfm", n_steps=7, fft_size=2048)),
        (20, 30000, 1, dict(method="essfm", n_steps=3, n_taps=8, fft_size=4096, boundary="zero")),
        (40, 40000, 2, dict(method="ssfm", n_steps=4, fft_size=8192)),
        (40, 33333, 1, dict(method="essfm", n_steps=1, n_taps=32, fft_size=8192)),
    ]
    plans, ins, outs, refs, kws = [], [], [], [], []
    for k, (spans, n, nw, kw) in enumerate(specs):
        kw = dict(kw)
        nc = kw.get("n_taps", 0)
        if nc:
            c = 0.6 * np.exp(-np.arange(nc + 1) / 5.0)
            kw["coeffs"] = (c / (c[0] + 2 * c[1:].sum())).astype(np.float32)
        p = Plan(synth.link(spans), FS, n, n_waveforms=nw, **kw)
        x = torch.from_numpy(synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=700 + k).astype(np.complex64)).cuda()
        plans.append(p)
        ins.append(x)
        outs.append(torch.zeros_like(x))
        refs.append(p.run(x))
        kws.append((synth.link(spans), kw))
    with Batch(plans, ins, outs) as batch:
        batch.run()
        assert batch.status() == 0
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for p, x, y, r, (link, kw) in zip(plans, ins, outs, refs, kws):
        assert torch.equal(y, r), kw
        info = p.info
        c = kw.get("coeffs")
        cfg = fiber.make_config(link, FS, kw["n_steps"], kw.get("n_taps", 0), kw["fft_size"],
                                coeffs=None if c is None else c.astype(np.float64), overlap=info.overlap,
                                boundary=kw.get("boundary", "periodic"), essfm=kw["method"] == "essfm")
        xs, ys = x.cpu().numpy(), y.cpu().numpy()
        n, v = xs.shape[-1], info.valid
        ids = np.unique(np.concatenate([[0, info.n_blocks - 1], rng.integers(0, info.n_blocks, 2)]))
        ref = odbp.dbp_blocks(xs[-1].astype(np.complex128), cfg, ids)
        for j, b in enumerate(ids):
            lo, hi = b * v, min((b + 1) * v, n)
            got = ys[-1][:, lo:hi].astype(np.complex128)
            want = ref[j][:, : hi - lo]
            rms = np.sqrt(np.mean(np.abs(want) ** 2))
            assert np.sqrt(np.mean(np.abs(got - want) ** 2)) / rms <= 1e-5, (kw, b)
            assert np.max(np.abs(got - want)) / rms <= 1e-4, (kw, b)
    for p in plans:
        p.close()
