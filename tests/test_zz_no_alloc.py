"""dbp_run_noalloc: the entry point for callers that cannot allocate device memory
(a host that must stay within pre-reserved buffers, an application whose allocator must
not be re-entered, a real-time loop that cannot afford an allocation's synchronisation).
It must give exactly what dbp_plan + dbp_run give (the same kernels on tables built by
the same kernels), on consecutive calls that reuse its one fixed scratch area, allocate
no device memory, and refuse problems that do not fit that scratch.  Called through the
C ABI with ctypes."""
import ctypes as C

import numpy as np
import pytest

import synth
from paper_1507_00921_gb300 import _lib
from paper_1507_00921_gb300.dbp import _Args

FS = synth.SAMPLE_RATE


def _args(spans, n, nw, **kw):
    kw.setdefault("coeffs", None)
    return _Args(synth.link(spans), FS, n, nw, kw.pop("boundary", "periodic"), kw.pop("method"),
                 kw.pop("n_steps"), kw.pop("n_taps", 0), kw.pop("coeffs"), kw.pop("coeffs_per_step", False),
                 kw.pop("step_len_m", None), kw.pop("gamma_eff", None), kw.pop("fft_size"), kw.pop("overlap", 0))


def _noalloc(lib, a, x_ptr, y_ptr, stream=0):
    return lib.dbp_run_noalloc(C.byref(a.link), C.byref(a.signal), C.byref(a.steps), C.c_void_p(x_ptr),
                               C.c_void_p(y_ptr), C.c_void_p(stream))


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = _lib.load()
    x = C.c_void_p(16)
    y = C.c_void_p(1 << 40)
    too_many = _args(40, 4096, 1, method="ssfm", n_steps=_lib.DBP_NOALLOC_MAX_STEPS + 1, fft_size=8192)
    assert lib.dbp_run_noalloc(C.byref(too_many.link), C.byref(too_many.signal), C.byref(too_many.steps), x, y,
                               None) == _lib.DBP_ERR_SCRATCH
    dz = np.linspace(0.5, 1.5, 20)
    dz = dz / dz.sum() * 3.2e6                      # 20 distinct step lengths: 20 H tables at N = 8192
    big = _args(40, 4096, 1, method="ssfm", n_steps=20, step_len_m=dz, fft_size=8192)
    assert lib.dbp_run_noalloc(C.byref(big.link), C.byref(big.signal), C.byref(big.steps), x, y,
                               None) == _lib.DBP_ERR_SCRATCH
    assert lib.dbp_strerror(_lib.DBP_ERR_SCRATCH) != b"unknown error"
    assert lib.dbp_run_noalloc(None, None, None, None, None, None) == _lib.DBP_ERR_ARG


@pytest.mark.gpu
def test_noalloc_matches_planned_run_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_00921_gb300 import Plan
    lib = _lib.load()
    c32 = 0.6 * np.exp(-np.arange(33) / 10.0)
    c32 = (c32 / (c32[0] + 2 * c32[1:].sum())).astype(np.float32)
    calls = [
        (40, 3 * 6760 + 11, 2, dict(method="essfm", n_steps=1, n_taps=32, coeffs=c32, fft_size=8192)),
        (10, 20000, 3, dict(method="ssfm", n_steps=5, fft_size=2048, boundary="zero")),
        (40, 12000, 1, dict(method="essfm", n_steps=3, n_taps=4, fft_size=4096,
                            step_len_m=np.array([0.5e6, 1.2e6, 1.5e6]),
                            coeffs=np.array([0.5, 0.2, 0.05, 0.01, 0.0], dtype=np.float32))),
    ]
    stream = torch.cuda.current_stream()
    # the first call on the device does the one-time set-up (scratch address lookup,
    # loading of the kernels); what follows must leave device memory untouched
    x0 = torch.zeros(2, 2, 4096, dtype=torch.complex64, device="cuda")
    y0 = torch.empty_like(x0)
    a0 = _args(10, 4096, 2, method="ssfm", n_steps=2, fft_size=1024)
    assert _noalloc(lib, a0, x0.data_ptr(), y0.data_ptr(), stream.cuda_stream) == _lib.DBP_OK
    torch.cuda.synchronize()
    for spans, n, nw, kw in calls:
        x = torch.from_numpy(synth.random_field(nw, n, synth.dbm_to_w(2.0), seed=n).astype(np.complex64)).cuda()
        kw2 = dict(kw)
        with Plan(synth.link(spans), FS, n, n_waveforms=nw, **kw2) as plan:
            ref = plan.run(x)
            torch.cuda.synchronize()
        a = _args(spans, n, nw, **dict(kw))
        y = torch.full_like(x, float("nan"))
        first = torch.empty_like(x)       # allocated before the measurement starts
        torch.cuda.synchronize()
        # Nothing that may allocate runs between the two readings of device memory: no
        # comparison (torch.equal allocates its result, and in a fresh process that can
        # make PyTorch's allocator reserve a new segment), only the two calls and copies
        # into buffers that already exist.
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        for k in range(2):   # two calls in a row on the shared scratch
            rc = _noalloc(lib, a, x.data_ptr(), y.data_ptr(), stream.cuda_stream)
            assert rc == _lib.DBP_OK, lib.dbp_strerror(rc)
            if k == 0:
                first.copy_(y)
                y.fill_(float("nan"))
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        alloc1 = torch.cuda.memory_allocated()
        assert free1 == free0
        assert alloc1 == alloc0
        assert torch.equal(first, ref)
        assert torch.equal(y, ref)
