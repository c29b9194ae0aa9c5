"""Out-of-memory paths, by host-side injection (no GPU fault): with
SOFT_TEST_ALLOC_BUDGET=N set when a plan is created, that plan's (N+1)-th
device allocation fails as out of memory.  Each failing call must return
SOFT_ERR_OUT_OF_MEMORY, free what it allocated (the library's live
allocation count comes back once the plan is gone), and leave the context
usable: the next plan, created without the hook, is correct."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, capi, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
ENV = "SOFT_TEST_ALLOC_BUDGET"


@pytest.fixture(autouse=True)
def _clean_env():
    torch.cuda.set_device(DEV)
    os.environ.pop(ENV, None)
    yield
    os.environ.pop(ENV, None)


def _create(B, dtype):
    lib = capi.load()
    h = ctypes.c_void_p()
    st = lib.soft_plan_create(ctypes.byref(h), B, dtype)
    return st, h


def _creation_budget(B, dtype):
    """Smallest budget with which soft_plan_create succeeds; every smaller one
    must fail with SOFT_ERR_OUT_OF_MEMORY, a NULL handle and no leak."""
    lib = capi.load()
    live0 = capi.soft_live_allocations()
    for n in range(64):
        os.environ[ENV] = str(n)
        st, h = _create(B, dtype)
        if st == capi.SOFT_OK:
            assert lib.soft_destroy(h) == capi.SOFT_OK
            assert capi.soft_live_allocations() == live0
            return n
        assert st == capi.SOFT_ERR_OUT_OF_MEMORY, (n, capi.status_string(st))
        assert not h.value
        assert capi.soft_live_allocations() == live0, n
        assert lib.soft_last_error()
    raise AssertionError("plan creation never succeeded")


@pytest.mark.parametrize("dtype", [capi.SOFT_FP64, capi.SOFT_MIXED_BF16X3, capi.SOFT_FP64_TC])
def test_plan_create_out_of_memory_at_every_allocation(dtype):
    assert _creation_budget(16, dtype) >= 10


def test_host_entry_point_and_correlate_out_of_memory():
    lib = capi.load()
    B = 16
    live0 = capi.soft_live_allocations()
    C = _creation_budget(B, capi.SOFT_FP64)
    grid = synth.random_grid(B, seed=8100)
    coef_out = np.zeros(synth.num_coeffs(B), dtype=np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    # the first staging buffer fails
    os.environ[ENV] = str(C)
    st, h = _create(B, capi.SOFT_FP64)
    assert st == capi.SOFT_OK
    st = lib.soft_forward_host(h, grid.ctypes.data_as(dp), coef_out.ctypes.data_as(dp), None)
    assert st == capi.SOFT_ERR_OUT_OF_MEMORY
    assert b"staging" in lib.soft_last_error()
    assert lib.soft_destroy(h) == capi.SOFT_OK
    assert capi.soft_live_allocations() == live0
    # the second staging buffer fails (the first stays with the plan until it is destroyed)
    os.environ[ENV] = str(C + 1)
    st, h = _create(B, capi.SOFT_FP64)
    assert st == capi.SOFT_OK
    assert lib.soft_inverse_host(h, coef_out.ctypes.data_as(dp), grid.ctypes.data_as(dp), None) == \
        capi.SOFT_ERR_OUT_OF_MEMORY
    assert lib.soft_destroy(h) == capi.SOFT_OK
    assert capi.soft_live_allocations() == live0
    # the correlation workspace fails
    os.environ[ENV] = str(C)
    st, h = _create(B, capi.SOFT_FP64)
    assert st == capi.SOFT_OK
    f_sh = torch.from_numpy(synth.sh_coefficients(B, seed=1)).to(DEV)
    g_sh = torch.from_numpy(synth.sh_coefficients(B, seed=2)).to(DEV)
    out = torch.empty((2 * B,) * 3, dtype=torch.complex128, device=DEV)
    st = lib.soft_correlate(h, f_sh.data_ptr(), g_sh.data_ptr(), out.data_ptr(), None, None, None)
    assert st == capi.SOFT_ERR_OUT_OF_MEMORY
    assert b"correlation workspace" in lib.soft_last_error()
    assert lib.soft_destroy(h) == capi.SOFT_OK
    assert capi.soft_live_allocations() == live0
    # without the hook, a fresh plan runs the same calls correctly
    os.environ.pop(ENV)
    with Plan(B, device=DEV) as p:
        got = p.forward_host(grid)
        corr, _, _ = p.correlate(f_sh, g_sh)
        p.sync()
        corr = corr.cpu().numpy()
    assert synth.rel_l2(got, oracle.forward(B, grid)) < 1e-10
    want = oracle.correlation(B, f_sh.cpu().numpy(), g_sh.cpu().numpy())
    assert synth.rel_l2(corr, want) < 1e-10
    assert capi.soft_live_allocations() == live0
