"""The FP64 plans' slice FFTs (the library's own radix-4 FFT for power-of-two
2B, cuFFT Z2Z otherwise) against the oracle, at a bound tighter than the
path's 1e-10: with FP64 on both sides the two differ only in the order of
rounding, ~log2(n) * 2^-53 per FFT and ~1e-14 through the whole transform,
so rel-L2 <= 1e-12 leaves a 40x margin and still catches a wrong twiddle
(which gives O(1)) or a twiddle of reduced precision (~1e-8 for FP32).

The DWT-only entry points isolate the FFT: the forward of the grid must match
the oracle's forward, and the DWT of the oracle's S (no FFT on the GPU) must
match it equally well, so any extra error comes from the GPU's FFT.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TIGHT = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


POW2_B = [1, 2, 4, 8, 16, 32, 64, 128]
OTHER_B = [3, 5, 12, 33]


@pytest.mark.parametrize("B", POW2_B + OTHER_B)
def test_forward_fft_step_is_fp64_accurate(B):
    grid = synth.random_grid(B, seed=7100 + B)
    want = oracle.forward(B, grid)
    with Plan(B, device=DEV) as p:
        full = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
        dwt_only = p.dwt_forward(torch.from_numpy(oracle.dft2_slices(grid, +1)).to(DEV)).cpu().numpy()
        p.sync()
    e_full, e_dwt = synth.rel_l2(full, want), synth.rel_l2(dwt_only, want)
    assert np.isfinite(full).all()
    assert e_full < TIGHT, (e_full, e_dwt)
    assert e_dwt < TIGHT


@pytest.mark.parametrize("B", POW2_B + OTHER_B)
def test_inverse_fft_step_is_fp64_accurate(B):
    coef = synth.coefficients(B, "gauss_decay", seed=7200 + B)
    want = oracle.inverse(B, coef)
    with Plan(B, device=DEV) as p:
        full = p.inverse(torch.from_numpy(coef).to(DEV)).cpu().numpy()
        s = p.dwt_inverse(torch.from_numpy(coef).to(DEV)).cpu().numpy()
        p.sync()
    e_full = synth.rel_l2(full, want)
    e_dwt = synth.rel_l2(oracle.dft2_slices(s, -1), want)
    assert np.isfinite(full).all()
    assert e_full < TIGHT, (e_full, e_dwt)
    assert e_dwt < TIGHT


@pytest.mark.parametrize("B", [8, 64])
def test_fft_of_one_plane_wave_per_slice(B):
    """A grid that is one plane wave exp(-i(m alpha + m' gamma)) per beta slice,
    a different (m, m') per slice: the + transform of each slice has a single
    nonzero entry, (2B)^2 at (m, m'), so a twiddle or bit-reversal slip moves
    energy to other entries and the sparse coefficient vector shows it."""
    n = 2 * B
    rng = np.random.default_rng(7300 + B)
    ms = rng.integers(1 - B, B, size=(n, 2))
    a = 2 * np.pi * np.arange(n) / n
    grid = np.empty((n, n, n), dtype=np.complex128)
    for j in range(n):
        m, mp = ms[j]
        grid[j] = np.exp(-1j * (m * a[:, None] + mp * a[None, :]))
    want = oracle.forward(B, grid)
    with Plan(B, device=DEV) as p:
        got = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(got, want) < TIGHT
