"""ctypes binding of libdbp (include/dbp.h): argument marshalling only.

Every computation happens inside the library's CUDA kernels; this module declares
the C structs and prototypes, loads the in-tree ``lib/libdbp.so`` (building it with
nvcc if it is missing or stale) and turns negative return codes into ``DBPError``.
There is no fallback: if the library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

DBP_OK = 0
DBP_ERR_ARG = -1
DBP_ERR_INFEASIBLE = -2
DBP_ERR_ALLOC = -3
DBP_ERR_CUDA = -4
DBP_ERR_TIMEOUT = -5
DBP_ERR_ALIAS = -6
DBP_ERR_UNSUPPORTED = -7
DBP_ERR_SCRATCH = -8
DBP_ERR_SINGULAR = -9
DBP_NOALLOC_SCRATCH_BYTES = 1 << 20
DBP_NOALLOC_MAX_STEPS = 64

DBP_PERIODIC, DBP_ZERO = 0, 1
DBP_SSFM, DBP_ESSFM, DBP_FFE = 0, 1, 2
DBP_SCHEME_FUSED, DBP_SCHEME_PER_STEP = 0, 1
DBP_FP32 = 0
DBP_SPLIT_BF16 = 1
DBP_SPLIT_FP16 = 2
DBP_MAX_TAPS = 64
DBP_BATCH_STREAMING = 1
DBP_MAX_STEPS = 1024


class dbp_link(C.Structure):
    _fields_ = [("n_spans", C.c_int32), ("span_len_m", C.c_double), ("alpha_db_per_km", C.c_double),
                ("D_ps_per_nm_km", C.c_double), ("lambda_m", C.c_double), ("gamma_per_W_km", C.c_double),
                ("manakov_factor", C.c_double)]


class dbp_signal(C.Structure):
    _fields_ = [("sample_rate_hz", C.c_double), ("n_samples", C.c_int64), ("n_waveforms", C.c_int32),
                ("boundary", C.c_int32), ("n_pols", C.c_int32)]


class dbp_steps(C.Structure):
    _fields_ = [("method", C.c_int32), ("n_steps", C.c_int32), ("n_taps", C.c_int32),
                ("coeffs", C.POINTER(C.c_float)), ("coeffs_per_step", C.c_int32),
                ("step_len_m", C.POINTER(C.c_double)), ("gamma_eff", C.POINTER(C.c_double)),
                ("fft_size", C.c_int32), ("overlap", C.c_int32), ("precision", C.c_int32),
                ("dft_block", C.c_int32), ("scheme", C.c_int32)]


class dbp_plan_info(C.Structure):
    _fields_ = [("fft_size", C.c_int32), ("overlap", C.c_int32), ("valid", C.c_int32), ("n_blocks", C.c_int32),
                ("n_steps", C.c_int32), ("n_taps", C.c_int32), ("beta2_s2_per_m", C.c_double),
                ("memory_samples", C.c_double), ("link_len_m", C.c_double)]


class DBPError(RuntimeError):
    def __init__(self, code: int, where: str, lib=None):
        msg = lib.dbp_strerror(code).decode() if lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


_P = C.c_void_p
_PROTOS = {
    "dbp_plan_describe": (C.c_int, [C.POINTER(dbp_link), C.POINTER(dbp_signal), C.POINTER(dbp_steps),
                                    C.POINTER(dbp_plan_info), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dbp_plan": (C.c_int, [C.POINTER(dbp_link), C.POINTER(dbp_signal), C.POINTER(dbp_steps), C.POINTER(_P)]),
    "dbp_plan_get_info": (C.c_int, [_P, C.POINTER(dbp_plan_info)]),
    "dbp_set_coeffs": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "dbp_run": (C.c_int, [_P, _P, _P, _P]),
    "dbp_run_host": (C.c_int, [_P, _P, _P, _P]),
    "dbp_grad": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "dbp_set_steps": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dbp_fit_coeffs": (C.c_int, [_P, _P, _P, C.c_longlong, C.c_int, C.c_double, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int), _P]),
    "dbp_run_noalloc": (C.c_int, [C.POINTER(dbp_link), C.POINTER(dbp_signal), C.POINTER(dbp_steps), _P, _P, _P]),
    "dbp_plan_status": (C.c_int, [_P]),
    "dbp_destroy": (None, [_P]),
    "dbp_batch_create": (C.c_int, [C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.c_int, C.c_int, C.c_int,
                                   C.POINTER(_P)]),
    "dbp_batch_run": (C.c_int, [_P, _P]),
    "dbp_batch_publish": (C.c_int, [_P, C.c_int, _P]),
    "dbp_batch_status": (C.c_int, [_P]),
    "dbp_batch_destroy": (None, [_P]),
    "dbp_run_batch": (C.c_int, [C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.c_int, _P]),
    "dbp_strerror": (C.c_char_p, [C.c_int]),
    "dbp_version": (C.c_char_p, []),
    "dbp_diag_fma": (C.c_int, [_P, C.c_int, C.c_int, _P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load (and if needed build) libdbp; raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and not _build.up_to_date():
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libdbp not built: {path}")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(code: int, where: str):
    if code != DBP_OK:
        raise DBPError(code, where, _lib)
