"""The host-buffer entry points (soft_forward_host / soft_inverse_host).

With the library's own slice FFT (FP64 and FP64-TC plans with power-of-two
2B) they pipeline the grid's host copies with the FFTs in chunks of beta
slices on a second stream; otherwise they copy, transform and copy back in
sequence.  Every slice's FFT is computed exactly as in the device-pointer call,
so the results must be bit-identical to it, for pageable and pinned host
buffers alike, and within the mode's bound of the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
BOUND = {"fp64": 1e-10, "fp64_tc": 1e-10, "bf16x3": 5e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _host_buffer(shape, pinned):
    if pinned:
        return torch.empty(shape, dtype=torch.complex128, pin_memory=True).numpy()
    return np.empty(shape, dtype=np.complex128)


# pipelined: power-of-two 2B in fp64 / fp64_tc, one chunk of slices for grids
# below 8 MiB (fp64) or 32 MiB (fp64_tc), 4 chunks for fp64 at B = 64, 8 at
# B = 128; sequential: cuFFT sizes and the FP32 modes
CASES = [(1, "fp64"), (2, "fp64"), (4, "fp64"), (32, "fp64"), (64, "fp64"), (3, "fp64"), (33, "fp64"),
         (2, "fp64_tc"), (16, "fp64_tc"), (64, "fp64_tc"), (128, "fp64_tc"), (12, "fp64_tc"), (16, "bf16x3")]


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("B,mode", CASES)
def test_host_calls_equal_device_calls(B, mode, pinned):
    n = 2 * B
    grid = synth.random_grid(B, seed=7400 + B)
    coef = synth.coefficients(B, "gauss_decay", seed=7500 + B)
    g_in = _host_buffer(grid.shape, pinned)
    g_in[...] = grid
    c_in = _host_buffer(coef.shape, pinned)
    c_in[...] = coef
    f_out = _host_buffer(coef.shape, pinned)
    f_out[...] = np.nan
    g_out = _host_buffer((n, n, n), pinned)
    g_out[...] = np.nan
    with Plan(B, mode, device=DEV) as p:
        f_dev = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
        g_dev = p.inverse(torch.from_numpy(coef).to(DEV)).cpu().numpy()
        p.forward_host(g_in, out=f_out)
        p.inverse_host(c_in, out=g_out)
        p.sync()
    assert np.array_equal(f_out, f_dev)
    assert np.array_equal(g_out, g_dev)
    assert np.array_equal(g_in, grid) and np.array_equal(c_in, coef), "a host call modified its input"
    assert synth.rel_l2(f_out, oracle.forward(B, grid)) < BOUND[mode]
    assert synth.rel_l2(g_out, oracle.inverse(B, coef)) < BOUND[mode]


@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_back_to_back_host_calls(mode):
    """Alternating host calls reuse the staging buffers and the copy stream:
    each result must still be the device call's on the same input (B = 128:
    8 chunks of slices)."""
    B = 128
    with Plan(B, mode, device=DEV) as p:
        for r in range(4):
            grid = synth.random_grid(B, seed=7600 + r)
            coef = synth.coefficients(B, "uniform", seed=7700 + r)
            f_host = p.forward_host(grid)
            g_host = p.inverse_host(coef)
            f_dev = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
            g_dev = p.inverse(torch.from_numpy(coef).to(DEV)).cpu().numpy()
            assert np.array_equal(f_host, f_dev), r
            assert np.array_equal(g_host, g_dev), r
        p.sync()
