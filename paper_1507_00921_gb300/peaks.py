"""Measured FP32 (non-tensor) FMA peak of the current GPU, via libdbp's diagnostic
kernel, for reporting the FP32-pipe utilisation of the DBP kernels."""
from __future__ import annotations

import ctypes as C


def fp32_fma_peak_tflops(iters: int = 4096, waves: int = 8, reps: int = 5) -> dict:
    import torch
    from . import _lib
    lib = _lib.load()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * waves
    out = torch.zeros(blocks * 256, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    _lib.check(lib.dbp_diag_fma(C.c_void_p(out.data_ptr()), blocks, 16, C.c_void_p(st.cuda_stream)), "fma")
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _lib.check(lib.dbp_diag_fma(C.c_void_p(out.data_ptr()), blocks, iters, C.c_void_p(st.cuda_stream)),
                   "fma")
        e1.record(st)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = max(best, blocks * 256 * iters * 256 / t / 1e12)
    return {"fp32_tflops": best, "sms": sms, "blocks": blocks, "iters": iters}


if __name__ == "__main__":
    import json
    print(json.dumps(fp32_fma_peak_tflops()))
