"""ctypes binding of the C ABI in include/soft.h, with the same names.

Argument marshalling only: every step of a transform runs in the CUDA
library.  Loading fails loudly if the library has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH

SOFT_OK = 0
SOFT_ERR_INVALID_ARG = 1
SOFT_ERR_OUT_OF_MEMORY = 2
SOFT_ERR_CUDA = 3
SOFT_ERR_UNSUPPORTED = 4
SOFT_ERR_TIMEOUT = 5
SOFT_ERR_DEVICE = 6

SOFT_FP64 = 0
SOFT_MIXED_BF16X3 = 1
SOFT_MIXED_TF32 = 2
SOFT_FP64_TC = 3

# name -> (restype, argtypes); mirrors include/soft.h
_vp, _i, _i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "soft_max_bandwidth": (_i, []),
    "soft_launch_count": (ctypes.c_ulonglong, []),
    "soft_live_allocations": (ctypes.c_longlong, []),
    "soft_num_coeffs": (_i64, [_i]),
    "soft_coef_index": (_i64, [_i, _i, _i, _i]),
    "soft_status_string": (ctypes.c_char_p, [_i]),
    "soft_last_error": (ctypes.c_char_p, []),
    "soft_plan_create": (_i, [ctypes.POINTER(_vp), _i, _i]),
    "soft_destroy": (_i, [_vp]),
    "soft_plan_bandwidth": (_i, [_vp]),
    "soft_plan_sync": (_i, [_vp]),
    "soft_forward": (_i, [_vp, _vp, _vp, _vp]),
    "soft_inverse": (_i, [_vp, _vp, _vp, _vp]),
    "soft_forward_real": (_i, [_vp, _vp, _vp, _vp]),
    "soft_inverse_real": (_i, [_vp, _vp, _vp, _vp]),
    "soft_forward_adjoint": (_i, [_vp, _vp, _vp, _vp]),
    "soft_inverse_adjoint": (_i, [_vp, _vp, _vp, _vp]),
    "soft_batched_inverse": (_i, [_i, _vp, _vp, _vp, _vp]),
    "soft_batched_forward": (_i, [_i, _vp, _vp, _vp, _vp]),
    "soft_batched_correlate": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "soft_correlation_coeffs": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "soft_correlate": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "soft_argmax_real": (_i, [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]),
    "soft_argmax_scratch_doubles": (_i, []),
    "soft_dwt_forward": (_i, [_vp, _vp, _vp, _vp]),
    "soft_dwt_inverse": (_i, [_vp, _vp, _vp, _vp]),
    "soft_dwt_forward_noalloc": (_i, [_i, _vp, _vp, _vp]),
    "soft_cluster_shard": (_i, [_i, _i, _i, _vp, _vp]),
    "soft_cluster_columns": (_i, [_i, _vp, _vp]),
    "soft_dwt_forward_clusters": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "soft_dwt_inverse_clusters": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "soft_gather_columns": (_i, [_vp, _vp, _i, _i, _vp, _i, _vp, _vp]),
    "soft_scatter_columns": (_i, [_vp, _vp, _i, _i, _vp, _i, _vp, _vp]),
    "soft_slice_fft": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "soft_forward_host": (_i, [_vp, _vp, _vp, _vp]),
    "soft_inverse_host": (_i, [_vp, _vp, _vp, _vp]),
    "soft_selftest_bounded_wait": (_i, [_vp, _i, _vp]),
    "soft_plan_num_variants": (_i, [_vp, _i]),
    "soft_plan_set_variant": (_i, [_vp, _i, _i]),
    "soft_plan_enable_timing": (_i, [_vp, _i]),
    "soft_plan_read_timing": (_i, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


class SoftError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = load().soft_last_error().decode()
        super().__init__(f"{what}: {status_string(status)} ({status})" + (f" [{detail}]" if detail else ""))


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libsoft_gb300.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().soft_status_string(int(status)).decode()


def check(status: int, what: str) -> None:
    if status != SOFT_OK:
        raise SoftError(status, what)


# Thin wrappers with the C names (pointers and streams as Python ints).
def soft_max_bandwidth() -> int:
    return load().soft_max_bandwidth()


def soft_launch_count() -> int:
    return int(load().soft_launch_count())


def soft_live_allocations() -> int:
    return int(load().soft_live_allocations())


def soft_num_coeffs(B: int) -> int:
    return load().soft_num_coeffs(B)


def soft_coef_index(B: int, l: int, m: int, mp: int) -> int:
    return load().soft_coef_index(B, l, m, mp)


def soft_plan_create(B: int, dtype: int = SOFT_FP64) -> int:
    h = ctypes.c_void_p()
    check(load().soft_plan_create(ctypes.byref(h), B, dtype), f"soft_plan_create(B={B}, dtype={dtype})")
    return h.value


def soft_destroy(plan: int | None) -> None:
    check(load().soft_destroy(plan), "soft_destroy")


def soft_plan_sync(plan: int) -> None:
    check(load().soft_plan_sync(plan), "soft_plan_sync")


def soft_forward(plan: int, grid_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    return load().soft_forward(plan, grid_ptr, coef_ptr, stream)


def soft_inverse(plan: int, coef_ptr: int, grid_ptr: int, stream: int = 0) -> int:
    return load().soft_inverse(plan, coef_ptr, grid_ptr, stream)


def soft_forward_real(plan: int, grid_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    return load().soft_forward_real(plan, grid_ptr, coef_ptr, stream)


def soft_inverse_real(plan: int, coef_ptr: int, grid_ptr: int, stream: int = 0) -> int:
    return load().soft_inverse_real(plan, coef_ptr, grid_ptr, stream)


def soft_forward_adjoint(plan: int, coef_ptr: int, grid_ptr: int, stream: int = 0) -> int:
    return load().soft_forward_adjoint(plan, coef_ptr, grid_ptr, stream)


def soft_inverse_adjoint(plan: int, grid_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    return load().soft_inverse_adjoint(plan, grid_ptr, coef_ptr, stream)


def soft_dwt_forward(plan: int, S_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    return load().soft_dwt_forward(plan, S_ptr, coef_ptr, stream)


def soft_dwt_inverse(plan: int, coef_ptr: int, S_ptr: int, stream: int = 0) -> int:
    return load().soft_dwt_inverse(plan, coef_ptr, S_ptr, stream)


def soft_dwt_forward_noalloc(B: int, S_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    """Forward DWT without a plan or any allocation (B <= 256); see include/soft.h."""
    return load().soft_dwt_forward_noalloc(B, S_ptr, coef_ptr, stream)


def soft_forward_host(plan: int, grid_ptr: int, coef_ptr: int, stream: int = 0) -> int:
    return load().soft_forward_host(plan, grid_ptr, coef_ptr, stream)


def soft_inverse_host(plan: int, coef_ptr: int, grid_ptr: int, stream: int = 0) -> int:
    return load().soft_inverse_host(plan, coef_ptr, grid_ptr, stream)


def soft_plan_enable_timing(plan: int, on: bool) -> None:
    check(load().soft_plan_enable_timing(plan, int(bool(on))), "soft_plan_enable_timing")


def soft_plan_read_timing(plan: int):
    """-> (ms[4], counts[4]) for {forward FFT, DWT, iDWT, inverse FFT} since the last read."""
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    check(load().soft_plan_read_timing(plan, ms, cnt), "soft_plan_read_timing")
    return list(ms), list(cnt)
