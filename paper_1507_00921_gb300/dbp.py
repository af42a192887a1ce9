"""Python front end of libdbp: plans and runs digital backpropagation on the GPU.

A ``Plan`` holds the link, signal and step parameters of Section II / III of
arXiv:1507.00921 (SSFM with N_s steps, or ESSFM with N_c filter coefficients) and the
device tables libdbp builds for them.  ``Plan.run`` takes a CUDA complex64 tensor
[n_waveforms, 2, n_samples] (or [2, n_samples]) and returns the backpropagated field;
every arithmetic step runs in libdbp's kernels on the tensor's device, on PyTorch's
current stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib

_BOUNDARY = {"periodic": _lib.DBP_PERIODIC, "zero": _lib.DBP_ZERO}
_METHOD = {"ssfm": _lib.DBP_SSFM, "essfm": _lib.DBP_ESSFM, "ffe": _lib.DBP_FFE}
_SCHEME = {"fused": _lib.DBP_SCHEME_FUSED, "per_step": _lib.DBP_SCHEME_PER_STEP}
_PRECISION = {"fp32": _lib.DBP_FP32, "split_bf16": _lib.DBP_SPLIT_BF16, "split_fp16": _lib.DBP_SPLIT_FP16}


def _link_struct(link: dict) -> _lib.dbp_link:
    return _lib.dbp_link(int(link["n_spans"]), float(link["span_len_m"]), float(link["alpha_db_per_km"]),
                         float(link["D_ps_per_nm_km"]), float(link["lambda_m"]), float(link["gamma_per_W_km"]),
                         float(link.get("manakov_factor", 1.0)))


@dataclass
class PlanInfo:
    fft_size: int
    overlap: int
    valid: int
    n_blocks: int
    n_steps: int
    n_taps: int
    beta2: float
    memory: float
    link_len_m: float
    step_dz: np.ndarray
    step_gamma_eff: np.ndarray


class _Args:
    """ctypes argument structs plus the host arrays they point into (kept alive)."""

    def __init__(self, link, fs, n_samples, n_waveforms, boundary, method, n_steps, n_taps, coeffs,
                 coeffs_per_step, step_len_m, gamma_eff, fft_size, overlap, precision="fp32", dft_block=0,
                 scheme="fused", n_pols=2):
        self.link = _link_struct(link)
        self.signal = _lib.dbp_signal(float(fs), int(n_samples), int(n_waveforms), _BOUNDARY[boundary],
                                      int(n_pols))
        self.coeffs = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float32)
        self.step_len = None if step_len_m is None else np.ascontiguousarray(step_len_m, dtype=np.float64)
        self.gamma_eff = None if gamma_eff is None else np.ascontiguousarray(gamma_eff, dtype=np.float64)
        fp = C.POINTER(C.c_float)
        dp = C.POINTER(C.c_double)
        self.steps = _lib.dbp_steps(
            _METHOD[method], int(n_steps), int(n_taps),
            self.coeffs.ctypes.data_as(fp) if self.coeffs is not None else fp(),
            int(bool(coeffs_per_step)),
            self.step_len.ctypes.data_as(dp) if self.step_len is not None else dp(),
            self.gamma_eff.ctypes.data_as(dp) if self.gamma_eff is not None else dp(),
            int(fft_size), int(overlap), _PRECISION[precision], int(dft_block), _SCHEME[scheme])


def describe(link: dict, fs: float, n_samples: int, *, n_waveforms=1, boundary="periodic", method="essfm",
             n_steps=1, n_taps=0, coeffs=None, coeffs_per_step=False, step_len_m=None, gamma_eff=None,
             fft_size=4096, overlap=0, precision="fp32", dft_block=0, scheme="fused", n_pols=2) -> PlanInfo:
    """Plan geometry and step table, computed by libdbp on the host (no GPU needed)."""
    lib = _lib.load()
    a = _Args(link, fs, n_samples, n_waveforms, boundary, method, n_steps, n_taps, coeffs, coeffs_per_step,
              step_len_m, gamma_eff, fft_size, overlap, precision, dft_block, scheme, n_pols)
    info = _lib.dbp_plan_info()
    dz = np.zeros(n_steps)
    ge = np.zeros(n_steps)
    dp = C.POINTER(C.c_double)
    rc = lib.dbp_plan_describe(C.byref(a.link), C.byref(a.signal), C.byref(a.steps), C.byref(info),
                               dz.ctypes.data_as(dp), ge.ctypes.data_as(dp))
    _lib.check(rc, "dbp_plan_describe")
    return PlanInfo(info.fft_size, info.overlap, info.valid, info.n_blocks, info.n_steps, info.n_taps,
                    info.beta2_s2_per_m, info.memory_samples, info.link_len_m, dz, ge)


class Plan:
    """A libdbp plan on the current CUDA device."""

    def __init__(self, link: dict, fs: float, n_samples: int, *, n_waveforms=1, boundary="periodic",
                 method="essfm", n_steps=1, n_taps=0, coeffs=None, coeffs_per_step=False, step_len_m=None,
                 gamma_eff=None, fft_size=4096, overlap=0, precision="fp32", dft_block=0, scheme="fused",
                 n_pols=2):
        """``n_pols=1``: one-polarization waveforms, complex64 [n_waveforms, n] (or
        [n_waveforms, 1, n]), the scalar ESSFM / SSFM with P_k = |y_k|^2."""
        import torch
        self._lib = _lib.load()
        self._args = _Args(link, fs, n_samples, n_waveforms, boundary, method, n_steps, n_taps, coeffs,
                           coeffs_per_step, step_len_m, gamma_eff, fft_size, overlap, precision, dft_block,
                           scheme, n_pols)
        self.n_samples = int(n_samples)
        self.n_waveforms = int(n_waveforms)
        self.n_pols = int(n_pols) if n_pols else 2
        self.method = method
        self.coeffs_per_step = bool(coeffs_per_step)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.info = describe(link, fs, n_samples, n_waveforms=n_waveforms, boundary=boundary, method=method,
                             n_steps=n_steps, n_taps=n_taps, coeffs=coeffs, coeffs_per_step=coeffs_per_step,
                             step_len_m=step_len_m, gamma_eff=gamma_eff, fft_size=fft_size, overlap=overlap,
                             precision=precision, dft_block=dft_block, scheme=scheme, n_pols=n_pols)
        h = C.c_void_p()
        rc = self._lib.dbp_plan(C.byref(self._args.link), C.byref(self._args.signal), C.byref(self._args.steps),
                                C.byref(h))
        _lib.check(rc, "dbp_plan")
        self._h = h
        self._coeffs = None if coeffs is None else np.array(coeffs, dtype=np.float32).ravel()

    # ------------------------------------------------------------------ helpers
    def _check_tensor(self, x, name):
        import torch
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.complex64:
            raise TypeError(f"{name} must be a CUDA complex64 tensor")
        if x.device != self.device:
            raise ValueError(f"{name} is on {x.device}, plan on {self.device}")
        want = (self.n_waveforms, self.n_pols, self.n_samples)
        if self.n_pols == 1:
            ok = x.numel() == np.prod(want) and x.shape[-1] == self.n_samples
        else:
            ok = x.numel() == np.prod(want) and x.shape[-2:] == (2, self.n_samples)
        if not ok:
            raise ValueError(f"{name} must have shape {want} (or [{self.n_pols}, n] for one waveform)")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")

    def run(self, x, out=None, stream=None):
        """Backpropagate x (CUDA complex64 [n_waveforms, 2, n]); returns ``out``."""
        import torch
        self._check_tensor(x, "x")
        if out is None:
            out = torch.empty_like(x)
        else:
            self._check_tensor(out, "out")
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        rc = self._lib.dbp_run(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                               C.c_void_p(st.cuda_stream))
        _lib.check(rc, "dbp_run")
        return out

    def run_host(self, x, out=None, stream=None):
        """Backpropagate a HOST complex64 array/tensor; copies in and out inside libdbp."""
        import torch
        xt = torch.as_tensor(x)
        if xt.is_cuda or xt.dtype != torch.complex64 or not xt.is_contiguous():
            raise TypeError("x must be a contiguous host complex64 array")
        if xt.numel() != self.n_waveforms * self.n_pols * self.n_samples:
            raise ValueError("x has the wrong number of samples")
        if out is None:
            out = torch.empty(xt.shape, dtype=torch.complex64, pin_memory=xt.is_pinned())
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        rc = self._lib.dbp_run_host(self._h, C.c_void_p(xt.data_ptr()), C.c_void_p(out.data_ptr()),
                                    C.c_void_p(st.cuda_stream))
        _lib.check(rc, "dbp_run_host")
        return out

    def grad(self, x, g_out, need_input=True, stream=None):
        """Reverse-mode gradient of ``run`` at input x for g_out = dL/dRe(out) + j dL/dIm(out).

        Returns ``(g_in, d_coeffs, d_gamma_eff, d_step_len)``: g_in (complex64, like x, or
        None), d_coeffs (float32 [n_steps, n_taps+1] if coeffs_per_step else [n_taps+1]),
        d_gamma_eff and d_step_len (float32 [n_steps]), all on the plan's device."""
        import torch
        self._check_tensor(x, "x")
        self._check_tensor(g_out, "g_out")
        ns, nt = self.info.n_steps, self.info.n_taps
        g_in = torch.empty_like(x) if need_input else None
        shape_c = (ns, nt + 1) if self.coeffs_per_step else (nt + 1,)
        d_c = torch.empty(shape_c, dtype=torch.float32, device=self.device)
        d_g = torch.empty(ns, dtype=torch.float32, device=self.device)
        d_z = torch.empty(ns, dtype=torch.float32, device=self.device)
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        rc = self._lib.dbp_grad(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(g_out.data_ptr()),
                                C.c_void_p(g_in.data_ptr() if g_in is not None else 0), C.c_void_p(d_c.data_ptr()),
                                C.c_void_p(d_g.data_ptr()), C.c_void_p(d_z.data_ptr()), C.c_void_p(st.cuda_stream))
        _lib.check(rc, "dbp_grad")
        return g_in, d_c, d_g, d_z

    def set_steps(self, step_len_m=None, gamma_eff=None):
        """Replace the step lengths (rebuilds H_s) and/or nonlinear strengths gamma_eff_s."""
        dp = C.POINTER(C.c_double)
        dz = None if step_len_m is None else np.ascontiguousarray(step_len_m, dtype=np.float64)
        ge = None if gamma_eff is None else np.ascontiguousarray(gamma_eff, dtype=np.float64)
        rc = self._lib.dbp_set_steps(self._h, dz.ctypes.data_as(dp) if dz is not None else dp(),
                                     ge.ctypes.data_as(dp) if ge is not None else dp())
        _lib.check(rc, "dbp_set_steps")
        if dz is not None:
            self.info.step_dz = dz.copy()
        if ge is not None:
            self.info.step_gamma_eff = ge.copy()

    def fit_coeffs(self, x, target, n_train=None, max_iter: int = 20, tol: float = 1e-12, coeffs0=None,
                   common_phase: bool = False, phase0: float = 0.0, stream=None):
        """Section IV least-squares fit of this single-step ESSFM plan's coefficients
        against ``target`` (same layout as ``x``; e.g. a many-step SSFM output), over the
        first ``n_train`` output samples of every waveform.  Gauss-Newton from ``coeffs0``
        (default the SSFM, c = 1, 0, ..., 0; c = 0 is the linear-only compensation).
        ``common_phase``: fit a common phase with the coefficients (what a receiver's
        carrier-phase recovery removes), starting at ``phase0``.  Returns ``(coeffs
        float64 [n_taps + 1], losses)``, or ``(coeffs, losses, phase)`` with
        ``common_phase``; losses are the mean |t - z|^2 per training vector sample at the
        start and after each update.  The plan's own coefficients are not changed."""
        import torch
        self._check_tensor(x, "x")
        self._check_tensor(target, "target")
        k = self.info.n_taps + 1
        c = np.zeros(k, dtype=np.float64)
        c[0] = 1.0
        if coeffs0 is not None:
            c[:] = np.asarray(coeffs0, dtype=np.float64).reshape(k)
        ph = np.array([float(phase0)], dtype=np.float64)
        losses = np.zeros(max_iter + 1, dtype=np.float64)
        n_iter = C.c_int(0)
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        dp = C.POINTER(C.c_double)
        rc = self._lib.dbp_fit_coeffs(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(target.data_ptr()),
                                      int(n_train or 0), int(max_iter), float(tol), c.ctypes.data_as(dp),
                                      ph.ctypes.data_as(dp) if common_phase else dp(), losses.ctypes.data_as(dp),
                                      C.byref(n_iter), C.c_void_p(st.cuda_stream))
        _lib.check(rc, "dbp_fit_coeffs")
        out = [float(v) for v in losses[:n_iter.value + 1]]
        return (c, out, float(ph[0])) if common_phase else (c, out)

    def set_coeffs(self, coeffs):
        c = np.ascontiguousarray(coeffs, dtype=np.float32)
        rc = self._lib.dbp_set_coeffs(self._h, c.ctypes.data_as(C.POINTER(C.c_float)))
        _lib.check(rc, "dbp_set_coeffs")
        self._coeffs = c.ravel().copy()

    def apply_params(self, coeffs=None, gamma_eff=None, step_len_m=None):
        """Makes the plan's coefficients, nonlinear strengths and step lengths equal to the
        given host arrays (None keeps the current value), uploading only what changed."""
        dz = None if step_len_m is None else np.asarray(step_len_m, dtype=np.float64).ravel()
        ge = None if gamma_eff is None else np.asarray(gamma_eff, dtype=np.float64).ravel()
        if dz is not None and np.array_equal(dz, self.info.step_dz):
            dz = None
        if ge is not None and np.array_equal(ge, self.info.step_gamma_eff):
            ge = None
        if dz is not None or ge is not None:
            self.set_steps(dz, ge)
        if coeffs is not None:
            c = np.asarray(coeffs, dtype=np.float32).ravel()
            if self._coeffs is None or not np.array_equal(c, self._coeffs):
                self.set_coeffs(c)

    def status(self):
        """Waits for the device; 0, or DBP_ERR_TIMEOUT if a bounded wait of the plan's
        tensor-core kernel gave up since the last call (the record is then cleared)."""
        return self._lib.dbp_plan_status(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dbp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many plans with their own device buffers, backpropagated by one CUDA-graph launch
    of persistent kernels (libdbp's dbp_batch_*).  Buffers must stay alive and in place."""

    def __init__(self, plans, ins, outs, streaming=False, timeout_us=0):
        self._lib = _lib.load()
        n = len(plans)
        if not (n == len(ins) == len(outs)) or n == 0:
            raise ValueError("plans, ins and outs must be non-empty lists of equal length")
        for pl, x, y in zip(plans, ins, outs):
            pl._check_tensor(x, "in")
            pl._check_tensor(y, "out")
        self._keep = (list(plans), list(ins), list(outs))
        arr = C.c_void_p * n
        self._p = arr(*[pl._h.value for pl in plans])
        self._i = arr(*[x.data_ptr() for x in ins])
        self._o = arr(*[y.data_ptr() for y in outs])
        h = C.c_void_p()
        rc = self._lib.dbp_batch_create(self._p, self._i, self._o, n,
                                        _lib.DBP_BATCH_STREAMING if streaming else 0, int(timeout_us), C.byref(h))
        _lib.check(rc, "dbp_batch_create")
        self._h = h

    def run(self, stream=None):
        import torch
        st = torch.cuda.current_stream() if stream is None else stream
        _lib.check(self._lib.dbp_batch_run(self._h, C.c_void_p(st.cuda_stream)), "dbp_batch_run")

    def publish(self, job, stream=None):
        import torch
        st = torch.cuda.current_stream() if stream is None else stream
        _lib.check(self._lib.dbp_batch_publish(self._h, int(job), C.c_void_p(st.cuda_stream)), "dbp_batch_publish")

    def status(self):
        """Waits for the device; returns 0 or a negative DBP_ERR_* code (e.g. timeout)."""
        return self._lib.dbp_batch_status(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.dbp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _autograd():
    import torch

    def host(t, dtype):
        return None if t is None else t.detach().to("cpu", dtype).numpy().copy()

    class DBPFunction(torch.autograd.Function):
        """out = DBP(x; c, gamma_eff, dz) through libdbp; backward through dbp_grad.

        ``DBPFunction.apply(x, coeffs, gamma_eff, step_len, plan)``: x the CUDA complex64
        waveforms, coeffs the ESSFM coefficients (shape of the plan's coefficient table),
        gamma_eff the per-step nonlinear strengths [n_steps] (1/W), step_len the per-step
        lengths [n_steps] (m) that set H_s (Eq. 1); any of the three may be None to keep
        the plan's current value.  The plan is brought to these values before the forward
        kernel and again before the adjoint (dbp_set_coeffs / dbp_set_steps; the block
        geometry and overlap stay those of the plan).  Returns the gradients of all four
        tensor inputs (Eqs. 1-3 differentiated by the adjoint kernel)."""

        @staticmethod
        def forward(ctx, x, coeffs, gamma_eff, step_len, plan):
            c = host(coeffs, torch.float32)
            ge = host(gamma_eff, torch.float64)
            dz = host(step_len, torch.float64)
            plan.apply_params(c, ge, dz)
            ctx.plan = plan
            ctx.params = (c, ge, dz)
            ctx.meta = [None if t is None else (t.device, t.dtype, t.shape) for t in (coeffs, gamma_eff, step_len)]
            ctx.save_for_backward(x)
            return plan.run(x.contiguous())

        @staticmethod
        def backward(ctx, g_out):
            (x,) = ctx.saved_tensors
            plan = ctx.plan
            plan.apply_params(*ctx.params)
            g_in, d_c, d_g, d_z = plan.grad(x, g_out.contiguous(), need_input=ctx.needs_input_grad[0])
            grads = []
            for g, meta, need in zip((d_c, d_g, d_z), ctx.meta, ctx.needs_input_grad[1:4]):
                grads.append(g.reshape(meta[2]).to(meta[0], meta[1]) if (meta is not None and need) else None)
            return (g_in, *grads, None)

    class DBP(torch.nn.Module):
        """ESSFM/SSFM backpropagation as a torch module over a Plan, with the coefficients
        c_{s,i}, the nonlinear strengths gamma_eff_s and the step lengths dz_s as
        parameters (by default only the coefficients are trained: gamma_eff and c trade
        off by a scale, and dz_s moves H_s)."""

        def __init__(self, plan, coeffs=None, gamma_eff=None, step_len_m=None, train_coeffs=True,
                     train_gamma_eff=False, train_step_len=False):
            super().__init__()
            nt = plan.info.n_taps
            shape = (plan.info.n_steps, nt + 1) if plan.coeffs_per_step else (nt + 1,)
            if coeffs is None:
                coeffs = np.zeros(shape, dtype=np.float32)
                coeffs[..., 0] = 1.0
            ge = plan.info.step_gamma_eff if gamma_eff is None else gamma_eff
            dz = plan.info.step_dz if step_len_m is None else step_len_m
            self.plan = plan
            self.coeffs = torch.nn.Parameter(torch.tensor(np.array(coeffs, dtype=np.float32)).reshape(shape),
                                             requires_grad=train_coeffs)
            self.gamma_eff = torch.nn.Parameter(torch.tensor(np.array(ge, dtype=np.float64)),
                                                requires_grad=train_gamma_eff)
            self.step_len = torch.nn.Parameter(torch.tensor(np.array(dz, dtype=np.float64)),
                                               requires_grad=train_step_len)

        def forward(self, x):
            return DBPFunction.apply(x, self.coeffs, self.gamma_eff, self.step_len, self.plan)

    return DBPFunction, DBP


def __getattr__(name):
    if name in ("DBPFunction", "DBP"):
        f, m = _autograd()
        return f if name == "DBPFunction" else m
    raise AttributeError(name)
