"""CPU checks of the C ABI: the library builds, loads, exports every symbol of
include/soft.h, and its host-only functions (sizes, layout, argument checks)
behave as documented.  No call here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1808_00896_gb300 import build as build_mod
from paper_1808_00896_gb300 import capi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return capi.load()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(soft_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in capi.SIGNATURES, f"binding lacks {n}"


def test_num_coeffs(lib):
    for B in (1, 2, 5, 64, 512):
        assert capi.soft_num_coeffs(B) == B * (4 * B * B - 1) // 3 == oracle.num_coeffs(B)
    assert capi.soft_num_coeffs(0) == -1


@pytest.mark.parametrize("B", [1, 2, 3, 6, 13])
def test_coef_index_matches_oracle_counting(lib, B):
    lmm = oracle.coef_lmm(B)
    for t, (l, m, mp) in enumerate(lmm):
        assert capi.soft_coef_index(B, int(l), int(m), int(mp)) == t
    assert capi.soft_coef_index(B, B, 0, 0) == -1
    assert capi.soft_coef_index(B, 0, 1, 0) == -1


def test_coef_index_large_B_sampled(lib):
    B = 512
    rng = np.random.default_rng(0)
    for _ in range(200):
        m, mp = (int(v) for v in rng.integers(1 - B, B, size=2))
        l0 = max(abs(m), abs(mp))
        l = int(rng.integers(l0, B))
        assert capi.soft_coef_index(B, l, m, mp) == oracle.coef_index(B, l, m, mp)
    assert capi.soft_coef_index(B, B - 1, B - 1, B - 1) == capi.soft_num_coeffs(B) - 1


def test_synth_degrees_match_layout(lib):
    B = 9
    ls = synth.coef_degrees(B)
    for t in range(0, len(ls), 7):
        l, m, mp = oracle.coef_lmm(B)[t]
        assert ls[t] == l and capi.soft_coef_index(B, int(l), int(m), int(mp)) == t


def test_plan_create_rejects_bad_arguments_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.soft_plan_create(ctypes.byref(h), 0, 0) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_plan_create(ctypes.byref(h), -3, 0) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_plan_create(ctypes.byref(h), capi.soft_max_bandwidth() + 1, 0) == capi.SOFT_ERR_UNSUPPORTED
    assert lib.soft_plan_create(ctypes.byref(h), 8, 7) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_plan_create(None, 8, 0) == capi.SOFT_ERR_INVALID_ARG
    assert h.value is None


def test_null_plan_handling(lib):
    assert lib.soft_destroy(None) == capi.SOFT_OK
    assert lib.soft_plan_bandwidth(None) == -1
    assert lib.soft_forward(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_inverse(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_plan_sync(None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_forward_real(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_inverse_real(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_forward_host(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_inverse_host(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert capi.status_string(capi.SOFT_ERR_TIMEOUT) == "SOFT_ERR_TIMEOUT"
    assert capi.status_string(99) == "SOFT_ERR_UNKNOWN"


def test_header_enums_match_the_binding():
    """Every SOFT_* enumerator of include/soft.h has the same value in capi."""
    import re
    header = open(os.path.join(os.path.dirname(__file__), "..", "include", "soft.h")).read()
    found = dict(re.findall(r"\b(SOFT_[A-Z0-9_]+)\s*=\s*(\d+)", header))
    assert {"SOFT_OK", "SOFT_FP64", "SOFT_MIXED_BF16X3", "SOFT_MIXED_TF32", "SOFT_FP64_TC",
            "SOFT_ERR_TIMEOUT", "SOFT_ERR_DEVICE"} <= set(found)
    for name, value in found.items():
        assert getattr(capi, name) == int(value), name


def test_launch_count_without_gpu(lib):
    """Calls rejected on the host launch nothing: the counter does not move."""
    c0 = capi.soft_launch_count()
    assert c0 >= 0
    assert lib.soft_forward(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert lib.soft_forward_real(None, None, None, None) == capi.SOFT_ERR_INVALID_ARG
    assert capi.soft_launch_count() == c0
