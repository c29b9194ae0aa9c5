"""GPU parity of the mixed-precision modes (contraction on tcgen05 tensor cores,
FP64 recurrence, FP32 2-D FFTs) against the FP64 CPU oracle.

Stated bounds (relative L2 error over all complex entries compared):
  BF16X3  <= 5e-5   products carry ~2^-16 relative error (hi = bf16_rn(x),
                    lo = bf16_rn(x - hi), the dropped lo*lo <= 2^-16), FP32
                    accumulation and FP32 FFTs add ~1e-7 each
  TF32    <= 2e-3   operands rounded to 10 explicit mantissa bits (2^-11)
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, capi, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
BOUND = {"bf16x3": 5e-5, "tf32": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def nan_coef(B):
    return torch.full((synth.num_coeffs(B),), complex(float("nan"), float("nan")), dtype=torch.complex128, device=DEV)


def nan_grid(B):
    n = 2 * B
    return torch.full((n, n, n), complex(float("nan"), float("nan")), dtype=torch.complex128, device=DEV)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
@pytest.mark.parametrize("B", [1, 2, 3, 8, 16, 17, 33, 64, 128])
def test_mixed_forward_parity(mode, B):
    coef = synth.coefficients(B, "gauss_decay", seed=8000 + B)
    grid = oracle.inverse(B, coef)  # band-limited input from the oracle
    with Plan(B, mode, device=DEV) as p:
        got = p.forward(torch.from_numpy(grid).to(DEV), out=nan_coef(B)).cpu().numpy()
        p.sync()
    assert np.isfinite(got).all()
    err = synth.rel_l2(got, oracle.forward(B, grid))
    assert err < BOUND[mode], f"{mode} B={B} forward rel-L2 {err:.3e}"


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
@pytest.mark.parametrize("B", [1, 2, 3, 8, 16, 17, 33, 64, 128])
def test_mixed_inverse_parity(mode, B):
    coef = synth.coefficients(B, "gauss_decay", seed=9000 + B)
    with Plan(B, mode, device=DEV) as p:
        got = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert np.isfinite(got).all()
    err = synth.rel_l2(got, oracle.inverse(B, coef))
    assert err < BOUND[mode], f"{mode} B={B} inverse rel-L2 {err:.3e}"


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_mixed_forward_on_raw_grid(mode):
    """Any grid (not band-limited): the quadrature sum of Eq. (quadrature)."""
    B = 32
    grid = synth.random_grid(B, seed=8500)
    with Plan(B, mode, device=DEV) as p:
        got = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
    assert synth.rel_l2(got, oracle.forward(B, grid)) < BOUND[mode]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
@pytest.mark.parametrize("B", [256, 512])
def test_mixed_sampled_parity_large(mode, B):
    rng = np.random.default_rng(B + 17)
    coef = synth.coefficients(B, "gauss_decay", seed=9500 + B)
    n = 2 * B
    with Plan(B, mode, device=DEV) as p:
        c = torch.from_numpy(coef).to(DEV)
        g = p.inverse(c)
        back = p.forward(g).cpu().numpy()
        p.sync()
        pts = [(0, 0, 0), (n - 1, 3, n - 2)] + [tuple(int(v) for v in rng.integers(0, n, size=3)) for _ in range(6)]
        g_pts = np.array([g[j, i, k].item() for (i, j, k) in pts])
    assert synth.rel_l2(g_pts, oracle.inverse_points(B, coef, pts)) < BOUND[mode]
    assert synth.rel_l2(back, coef) < 2 * BOUND[mode]


def test_mixed_plans_reject_fp64_step_entry_points():
    B = 8
    with Plan(B, "bf16x3", device=DEV) as p:
        S = torch.zeros((2 * B,) * 3, dtype=torch.complex128, device=DEV)
        c = torch.zeros(synth.num_coeffs(B), dtype=torch.complex128, device=DEV)
        lib = capi.load()
        assert lib.soft_dwt_forward(p.handle, S.data_ptr(), c.data_ptr(), None) == capi.SOFT_ERR_UNSUPPORTED
        assert lib.soft_dwt_inverse(p.handle, c.data_ptr(), S.data_ptr(), None) == capi.SOFT_ERR_UNSUPPORTED
