"""GPU parity of the FP64-accurate tensor-core mode (SOFT_FP64_TC: FP64
recurrence and S; contraction as exact base-128 BF16 digit products on
tcgen05; double-float 2-D FFTs) against the FP64 CPU oracle, at the FP64
path's bound.

Bound: relative L2 error <= 1e-10 over all complex entries compared, the same
as the plain FP64 path.  Derivation: each operand entry is carried to 2^-49
of its scale (7 digits of 7 bits, the leading one 6 bits plus sign); the
dropped digit pairs of level >= 7 and the two rounding residuals give a
product error of a few times 2^-49 of (row scale x column scale); the level
sums 0..3 are exact integers combined exactly, levels 4..6 carry FP32
rounding at weight <= 2^-28.  Entries are typically >= 1e-2 of their scales,
so the expected error is ~1e-12, two orders inside the bound (measured
1.6e-13 .. 5.5e-13).  The 2-D FFTs of power-of-two bandwidths run in
double-float arithmetic (~2^-47 per operation, norm-wise).

Outputs are pre-filled with NaN so that an entry the kernels never write
fails the comparison.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, batched_forward, batched_inverse, capi, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TOL = 1e-10
MODE = "fp64_tc"


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


SMALL_B = [1, 2, 3, 4, 5, 8, 11, 16, 17, 32, 33, 64]


@pytest.mark.parametrize("B", SMALL_B)
def test_forward_parity(B):
    grid = synth.random_grid(B, seed=21000 + B)
    with Plan(B, MODE, device=DEV) as p:
        got = p.forward(torch.from_numpy(grid).to(DEV), out=nan_coef(B)).cpu().numpy()
        p.sync()
    assert np.isfinite(got).all()
    err = synth.rel_l2(got, oracle.forward(B, grid))
    assert err < TOL, f"B={B} forward rel-L2 {err:.3e}"


@pytest.mark.parametrize("B", SMALL_B)
def test_inverse_parity(B):
    coef = synth.coefficients(B, "uniform", seed=22000 + B)
    with Plan(B, MODE, device=DEV) as p:
        got = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert np.isfinite(got).all()
    err = synth.rel_l2(got, oracle.inverse(B, coef))
    assert err < TOL, f"B={B} inverse rel-L2 {err:.3e}"


@pytest.mark.parametrize("B", [16, 64])
def test_band_limited_gauss_decay(B):
    """The smooth workload of the benchmark: inverse of 1/(l+1)-decaying
    coefficients, then forward back (the round trip is the identity)."""
    coef = synth.coefficients(B, "gauss_decay", seed=23000 + B)
    with Plan(B, MODE, device=DEV) as p:
        g = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B))
        back = p.forward(g, out=nan_coef(B)).cpu().numpy()
        g = g.cpu().numpy()
        p.sync()
    assert synth.rel_l2(g, oracle.inverse(B, coef)) < TOL
    assert synth.rel_l2(back, coef) < TOL


@pytest.mark.parametrize("B", [4, 16, 64])
def test_dwt_steps_alone(B):
    grid = synth.random_grid(B, seed=24000 + B)
    S = oracle.dft2_slices(grid, +1)
    coef = synth.coefficients(B, "gauss_decay", seed=24100 + B)
    with Plan(B, MODE, device=DEV) as p:
        f = p.dwt_forward(torch.from_numpy(S).to(DEV), out=nan_coef(B)).cpu().numpy()
        s_inv = p.dwt_inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, grid)) < TOL
    assert np.all(s_inv[:, B, :] == 0) and np.all(s_inv[:, :, B] == 0)
    assert synth.rel_l2(oracle.dft2_slices(s_inv, -1), oracle.inverse(B, coef)) < TOL


def test_full_parity_B128():
    B = 128
    grid = synth.random_grid(B, seed=25128)
    coef = synth.coefficients(B, "gauss_decay", seed=25129)
    with Plan(B, MODE, device=DEV) as p:
        f = p.forward(torch.from_numpy(grid).to(DEV), out=nan_coef(B)).cpu().numpy()
        g = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, grid)) < TOL
    assert synth.rel_l2(g, oracle.inverse(B, coef)) < TOL


@pytest.mark.parametrize("B", [80, 96])
def test_partial_second_sample_tile(B):
    """The inverse runs two 128-beta-sample tiles at a time; at 2B = 160 and 192
    the second tile of the pair is partly past the last sample (its idle lanes
    run on zeros and are not stored).  Full parity, both directions."""
    grid = synth.random_grid(B, seed=27000 + B)
    coef = synth.coefficients(B, "gauss_decay", seed=27100 + B)
    with Plan(B, MODE, device=DEV) as p:
        f = p.forward(torch.from_numpy(grid).to(DEV), out=nan_coef(B)).cpu().numpy()
        g = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, grid)) < TOL
    assert synth.rel_l2(g, oracle.inverse(B, coef)) < TOL


@pytest.mark.parametrize("B", [160, 192])
def test_odd_number_of_sample_tiles(B):
    """2B = 320 and 384: three 128-sample tiles, so the inverse's second pair
    has a second tile wholly (192) or partly (160) past the last sample.
    Every grid value of sampled beta slices in both pairs against the oracle's
    one-by-one sums, and the round trip."""
    rng = np.random.default_rng(B)
    coef = synth.coefficients(B, "gauss_decay", seed=27200 + B)
    n = 2 * B
    with Plan(B, MODE, device=DEV) as p:
        g = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B))
        back = p.forward(g).cpu().numpy()
        p.sync()
        # beta slices j in each tile, the last sample, and random (alpha, gamma) points
        js = [0, 127, 128, 255, 256, n - 1]
        pts = [(int(rng.integers(0, n)), j, int(rng.integers(0, n))) for j in js for _ in range(2)]
        g_pts = np.array([g[j, i, k].item() for (i, j, k) in pts])
    assert np.isfinite(g_pts).all()
    assert synth.rel_l2(g_pts, oracle.inverse_points(B, coef, pts)) < TOL
    assert synth.rel_l2(back, coef) < TOL


@pytest.mark.parametrize("B", [256, 512])
def test_sampled_parity_large(B):
    """Full-size bandwidths in the benchmark's launch configuration: forward
    coefficients of sampled order pairs and inverse values at sampled grid
    points against the oracle's one-by-one forms, plus the round trip."""
    rng = np.random.default_rng(B + 5)
    grid = synth.random_grid(B, seed=26000 + B)
    coef = synth.coefficients(B, "gauss_decay", seed=26100 + B)
    n = 2 * B
    with Plan(B, MODE, device=DEV) as p:
        f = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
        g = p.inverse(torch.from_numpy(coef).to(DEV))
        back = p.forward(g).cpu().numpy()
        p.sync()
        pts = [(0, 0, 0), (n - 1, n - 1, n - 1)] + [tuple(int(v) for v in rng.integers(0, n, size=3))
                                                   for _ in range(6)]
        g_pts = np.array([g[j, i, k].item() for (i, j, k) in pts])
    pairs = [(0, 0), (B - 1, B - 1), (1 - B, B - 1), (B - 1, 0), (0, 1 - B), (B // 2, B // 2), (-(B // 3), B // 5)]
    while len(pairs) < 10:
        pairs.append(tuple(int(v) for v in rng.integers(1 - B, B, size=2)))
    want = oracle.forward_pairs(B, grid, pairs)
    got = []
    for (m, mp) in pairs:
        l0 = max(abs(m), abs(mp))
        o = capi.soft_coef_index(B, l0, m, mp)
        got.append(f[o:o + B - l0])
    assert synth.rel_l2(np.concatenate(got), np.concatenate(want)) < TOL
    assert synth.rel_l2(g_pts, oracle.inverse_points(B, coef, pts)) < TOL
    assert synth.rel_l2(back, coef) < TOL


@pytest.mark.parametrize("B", [1, 3, 8, 16, 64])
def test_adjoint_parity(B):
    c = synth.coefficients(B, "uniform", seed=27000 + B)
    x = synth.random_grid(B, seed=28000 + B)
    with Plan(B, MODE, device=DEV) as p:
        fa = p.forward_adjoint(torch.from_numpy(c).to(DEV)).cpu().numpy()
        ia = p.inverse_adjoint(torch.from_numpy(x).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(fa, oracle.forward_adjoint(B, c)) < TOL
    assert synth.rel_l2(ia, oracle.inverse_adjoint(B, x)) < TOL


def test_agrees_with_plain_fp64_path():
    """Same inputs through the two FP64-accurate GPU modes."""
    B = 48
    grid = torch.from_numpy(synth.random_grid(B, seed=29000)).to(DEV)
    coef = torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=29001)).to(DEV)
    with Plan(B, "fp64", device=DEV) as a, Plan(B, MODE, device=DEV) as b:
        fa, fb = a.forward(grid).cpu().numpy(), b.forward(grid).cpu().numpy()
        ga, gb = a.inverse(coef).cpu().numpy(), b.inverse(coef).cpu().numpy()
    assert synth.rel_l2(fb, fa) < TOL
    assert synth.rel_l2(gb, ga) < TOL


def test_batched_mixes_fp64tc_with_other_modes():
    specs = [(16, MODE), (32, "fp64"), (16, "bf16x3"), (24, MODE)]
    plans = [Plan(B, m, device=DEV) for B, m in specs]
    try:
        coefs = [torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=29100 + i)).to(DEV)
                 for i, (B, _) in enumerate(specs)]
        grids = batched_inverse(plans, coefs)
        back = batched_forward(plans, grids)
        torch.cuda.synchronize(DEV)
        for (B, m), c, g, f in zip(specs, coefs, grids, back):
            bound = 5e-5 if m == "bf16x3" else TOL
            ref = oracle.inverse(B, c.cpu().numpy())
            assert synth.rel_l2(g.cpu().numpy(), ref) < bound
            assert synth.rel_l2(f.cpu().numpy(), c.cpu().numpy()) < 2 * bound
    finally:
        for p in plans:
            p.close()


def test_one_hot_coefficient_gives_wigner_D():
    """A single coefficient f(l,m,m') = 1 gives the Wigner D-function on the
    grid (the oracle's inverse of the same one-hot vector), including the
    largest degree and orders."""
    B = 40
    for (l, m, mp) in [(B - 1, B - 1, -(B - 1)), (B - 1, 0, 0), (17, -5, 12), (0, 0, 0)]:
        c = np.zeros(synth.num_coeffs(B), dtype=np.complex128)
        c[capi.soft_coef_index(B, l, m, mp)] = 1.0
        with Plan(B, MODE, device=DEV) as p:
            g = p.inverse(torch.from_numpy(c).to(DEV)).cpu().numpy()
            back = p.forward(torch.from_numpy(g).to(DEV)).cpu().numpy()
        assert synth.rel_l2(g, oracle.inverse(B, c)) < TOL
        assert synth.rel_l2(back, c) < TOL


@pytest.mark.parametrize("scale", [1e-150, 1e150])
def test_inputs_far_outside_the_fp32_range(scale):
    """The double-float FFT of power-of-two bandwidths works on the data scaled
    by the power of two of its largest magnitude, and the digit scales of the
    contraction come from the data too, so accuracy holds at any FP64 scale."""
    B = 16
    grid = synth.random_grid(B, seed=31000) * scale
    coef = synth.coefficients(B, "gauss_decay", seed=31001) * scale
    with Plan(B, MODE, device=DEV) as p:
        f = p.forward(torch.from_numpy(grid).to(DEV), out=nan_coef(B)).cpu().numpy()
        g = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, grid)) < TOL
    assert synth.rel_l2(g, oracle.inverse(B, coef)) < TOL


def test_all_zero_input():
    B = 8
    with Plan(B, MODE, device=DEV) as p:
        f = p.forward(torch.zeros((2 * B,) * 3, dtype=torch.complex128, device=DEV), out=nan_coef(B)).cpu().numpy()
        g = p.inverse(torch.zeros(synth.num_coeffs(B), dtype=torch.complex128, device=DEV), out=nan_grid(B))
        p.sync()
    assert np.all(f == 0)
    assert torch.all(g == 0)


def test_full_size_B512_against_the_fp64_path():
    """Every coefficient and every grid value at B = 512 (1024^3 grid) against
    the plain FP64 GPU path, whose own agreement with the oracle the sampled
    tests establish at this size.  Norms are taken on the device."""
    B = 512
    grid = torch.from_numpy(synth.random_grid(B, seed=32512)).to(DEV)
    coef = torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=32513)).to(DEV)

    def rel(x, ref):
        return (torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)).item()

    with Plan(B, "fp64", device=DEV) as a:
        fa = a.forward(grid)
        ga = a.inverse(coef)
        a.sync()
    with Plan(B, MODE, device=DEV) as b:
        fb = b.forward(grid)
        gb = b.inverse(coef)
        b.sync()
    del grid
    assert rel(fb, fa) < TOL
    assert rel(gb, ga) < TOL
