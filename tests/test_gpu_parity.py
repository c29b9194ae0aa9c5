"""GPU parity: the CUDA path (through the C ABI) vs the FP64 CPU oracle on the
same seeded inputs.  Tolerance for the FP64 path: relative L2 error <= 1e-10
over all complex entries compared (the bound stated for the FP64 path; both
sides run the same FP64 arithmetic in different orders, so the observed error
is ~1e-14).

Outputs are pre-filled with NaN so that an entry the kernels never write
fails the comparison.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, capi, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def nan_like_coef(B):
    return torch.full((synth.num_coeffs(B),), complex(float("nan"), float("nan")),
                      dtype=torch.complex128, device=DEV)


def nan_grid(B):
    n = 2 * B
    return torch.full((n, n, n), complex(float("nan"), float("nan")), dtype=torch.complex128, device=DEV)


SMALL_B = [1, 2, 3, 4, 5, 8, 11, 16, 17, 32, 33, 64]


@pytest.mark.parametrize("B", SMALL_B)
def test_forward_parity(B):
    grid = synth.random_grid(B, seed=1000 + B)
    g = torch.from_numpy(grid).to(DEV)
    with Plan(B, device=DEV) as p:
        out = p.forward(g, out=nan_like_coef(B))
        p.sync()
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert synth.rel_l2(got, oracle.forward(B, grid)) < TOL
    assert torch.equal(g.cpu(), torch.from_numpy(grid)), "forward modified its input"


@pytest.mark.parametrize("B", SMALL_B)
def test_inverse_parity(B):
    coef = synth.coefficients(B, "uniform", seed=2000 + B)
    c = torch.from_numpy(coef).to(DEV)
    with Plan(B, device=DEV) as p:
        out = p.inverse(c, out=nan_grid(B))
        p.sync()
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert synth.rel_l2(got, oracle.inverse(B, coef)) < TOL
    assert torch.equal(c.cpu(), torch.from_numpy(coef)), "inverse modified its input"


@pytest.mark.parametrize("B", [4, 16, 64])
def test_dwt_steps_alone(B):
    """soft_dwt_forward on the oracle's S = 2-D DFT(+) of each slice equals the
    oracle's forward; soft_dwt_inverse then the oracle's DFT(-) equals its inverse."""
    grid = synth.random_grid(B, seed=3000 + B)
    S = oracle.dft2_slices(grid, +1)
    coef = synth.coefficients(B, "gauss_decay", seed=3100 + B)
    with Plan(B, device=DEV) as p:
        f = p.dwt_forward(torch.from_numpy(S).to(DEV), out=nan_like_coef(B)).cpu().numpy()
        s_inv = p.dwt_inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, grid)) < TOL
    n = 2 * B
    assert np.all(s_inv[:, B, :] == 0) and np.all(s_inv[:, :, B] == 0)
    assert synth.rel_l2(oracle.dft2_slices(s_inv, -1), oracle.inverse(B, coef)) < TOL
    assert s_inv.shape == (n, n, n)


@pytest.mark.parametrize("B,kind", [(16, "uniform"), (64, "gauss_decay"), (128, "gauss_decay")])
def test_round_trip_on_band_limited(B, kind):
    coef = synth.coefficients(B, kind, seed=4000 + B)
    c = torch.from_numpy(coef).to(DEV)
    with Plan(B, device=DEV) as p:
        back = p.forward(p.inverse(c))
        p.sync()
    assert synth.rel_l2(back.cpu().numpy(), coef) < TOL


def test_full_parity_B128():
    B = 128
    grid = synth.random_grid(B, seed=5128)
    coef = synth.coefficients(B, "gauss_decay", seed=5129)
    with Plan(B, device=DEV) as p:
        f = p.forward(torch.from_numpy(grid).to(DEV), out=nan_like_coef(B)).cpu().numpy()
        g = p.inverse(torch.from_numpy(coef).to(DEV), out=nan_grid(B)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, grid)) < TOL
    assert synth.rel_l2(g, oracle.inverse(B, coef)) < TOL


def _sampled_pairs(B, rng, count):
    pairs = [(0, 0), (B - 1, B - 1), (1 - B, B - 1), (B - 1, 0), (0, 1 - B), (B // 2, B // 2),
             (-(B // 3), B // 5)]
    while len(pairs) < count:
        pairs.append(tuple(int(v) for v in rng.integers(1 - B, B, size=2)))
    return pairs


def _run(p, B, pair):
    l0 = max(abs(pair[0]), abs(pair[1]))
    o = capi.soft_coef_index(B, l0, pair[0], pair[1])
    return o, B - l0


@pytest.mark.parametrize("B", [256, 512])
def test_sampled_parity_large(B):
    """Full-size bandwidths, in the launch configuration the benchmark uses:
    forward coefficients of sampled order pairs and inverse values at sampled
    grid points against the oracle's one-by-one forms, plus the round trip."""
    rng = np.random.default_rng(B)
    grid = synth.random_grid(B, seed=6000 + B)
    coef = synth.coefficients(B, "gauss_decay", seed=6100 + B)
    with Plan(B, device=DEV) as p:
        f = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
        c = torch.from_numpy(coef).to(DEV)
        g = p.inverse(c)
        back = p.forward(g).cpu().numpy()
        p.sync()
        n = 2 * B
        pts = [(0, 0, 0), (n - 1, n - 1, n - 1)] + [tuple(int(v) for v in rng.integers(0, n, size=3))
                                                   for _ in range(6)]
        g_pts = np.array([g[j, i, k].item() for (i, j, k) in pts])
    pairs = _sampled_pairs(B, rng, 10 if B == 256 else 8)
    want = oracle.forward_pairs(B, grid, pairs)
    got = np.concatenate([f[o:o + L] for o, L in (_run(p, B, pr) for pr in pairs)])
    assert synth.rel_l2(got, np.concatenate(want)) < TOL
    assert synth.rel_l2(g_pts, oracle.inverse_points(B, coef, pts)) < TOL
    assert synth.rel_l2(back, coef) < TOL


def test_host_entry_points_match_device():
    B = 32
    grid = synth.random_grid(B, seed=7032)
    coef = synth.coefficients(B, "uniform", seed=7033)
    with Plan(B, device=DEV) as p:
        f_dev = p.forward(torch.from_numpy(grid).to(DEV)).cpu().numpy()
        g_dev = p.inverse(torch.from_numpy(coef).to(DEV)).cpu().numpy()
        f_host = p.forward_host(grid)
        g_host = p.inverse_host(coef)
    assert np.array_equal(f_dev, f_host)
    assert np.array_equal(g_dev, g_host)


def test_timing_counters():
    B = 16
    with Plan(B, device=DEV) as p:
        capi.soft_plan_enable_timing(p.handle, True)
        c = torch.from_numpy(synth.coefficients(B, "uniform", seed=1)).to(DEV)
        for _ in range(3):
            p.forward(p.inverse(c))
        ms, cnt = capi.soft_plan_read_timing(p.handle)
        assert cnt == [3, 3, 3, 3]
        assert all(v > 0 for v in ms)
        ms2, cnt2 = capi.soft_plan_read_timing(p.handle)
        assert cnt2 == [0, 0, 0, 0]


def test_argument_errors_on_gpu():
    B = 8
    with Plan(B, device=DEV) as p:
        g = torch.zeros((2 * B,) * 3, dtype=torch.complex128, device=DEV)
        c = torch.zeros(synth.num_coeffs(B), dtype=torch.complex128, device=DEV)
        lib = capi.load()
        h = p.handle
        assert lib.soft_forward(h, None, c.data_ptr(), None) == capi.SOFT_ERR_INVALID_ARG
        assert lib.soft_forward(h, g.data_ptr() + 8, c.data_ptr(), None) == capi.SOFT_ERR_INVALID_ARG
        assert lib.soft_inverse(h, c.data_ptr(), c.data_ptr(), None) == capi.SOFT_ERR_INVALID_ARG
        with pytest.raises(TypeError):
            p.forward(g.to(torch.complex64))
        with pytest.raises(ValueError):
            p.forward(c)
        assert lib.soft_plan_bandwidth(h) == B


def test_bounded_wait_reports_timeout_and_context_survives():
    """A wait that nothing satisfies gives up after its poll limit, the kernel
    records a timeout, soft_plan_sync reports it, and the next transform on the
    same context is still correct."""
    B = 8
    with Plan(B, "bf16x3", device=DEV) as p:
        lib = capi.load()
        assert lib.soft_selftest_bounded_wait(p.handle, 2000, None) == capi.SOFT_OK
        assert lib.soft_plan_sync(p.handle) == capi.SOFT_ERR_TIMEOUT
        assert lib.soft_plan_sync(p.handle) == capi.SOFT_OK  # the error word is cleared once read
        coef = synth.coefficients(B, "uniform", seed=77)
        g = p.inverse(torch.from_numpy(coef).to(DEV))
        p.sync()
        assert synth.rel_l2(g.cpu().numpy(), oracle.inverse(B, coef)) < 5e-5
        assert lib.soft_selftest_bounded_wait(p.handle, 0, None) == capi.SOFT_ERR_INVALID_ARG


def test_launch_count():
    """soft_launch_count: an FP64 forward with the library's FFT is 3 launches
    (rows and columns passes, DWT) and an inverse 4 (S clearing, iDWT, two FFT
    passes); with cuFFT (2B not a power of two) they are 1 and 2.  A batch's
    graph counts its kernels at every replay."""
    for B, fwd, inv in ((16, 3, 4), (3, 1, 2)):
        grid = torch.from_numpy(synth.random_grid(B, seed=7800 + B)).to(DEV)
        coef = torch.from_numpy(synth.coefficients(B, "uniform", seed=7900 + B)).to(DEV)
        with Plan(B, device=DEV) as p:
            c0 = capi.soft_launch_count()
            p.forward(grid)
            c1 = capi.soft_launch_count()
            p.inverse(coef)
            c2 = capi.soft_launch_count()
            p.sync()
        assert (c1 - c0, c2 - c1) == (fwd, inv), B
    from paper_1808_00896_gb300 import batched_inverse
    plans = [Plan(16, device=DEV) for _ in range(3)]
    coefs = [torch.from_numpy(synth.coefficients(16, "uniform", seed=8000 + i)).to(DEV) for i in range(3)]
    outs = [p.empty_grid() for p in plans]
    batched_inverse(plans, coefs, outs)  # captures the graph
    per = []
    for _ in range(3):
        c0 = capi.soft_launch_count()
        batched_inverse(plans, coefs, outs)
        per.append(capi.soft_launch_count() - c0)
    torch.cuda.synchronize(DEV)
    for p in plans:
        p.close()
    assert per[0] > 0 and per == [per[0]] * 3, per
