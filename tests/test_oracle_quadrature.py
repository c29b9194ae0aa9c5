"""Pins for the oracle's sampling grid, quadrature weights and DFTs
(Eq. (quadrature) and Eq. (weights) of the paper)."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("B", [1, 2, 3, 8, 17, 64, 512])
def test_weights_sum_and_symmetry(B):
    w = oracle.weights(B)
    assert w.shape == (2 * B,)
    assert abs(w.sum() - 2 * math.pi / B) < 1e-14 * (2 * math.pi / B) * 4 * B
    # mirror-equal up to rounding: sin(beta) near pi and the B-term sum lose a few digits
    assert np.max(np.abs(w - w[::-1])) < 1e-13 * np.max(w)
    assert np.all(w > 0)


@pytest.mark.parametrize("B", [1, 2, 4, 7, 16, 64])
def test_weights_integrate_legendre_exactly(B):
    """sum_j w_B(j) P_k(cos beta_j) = (pi/B) int_0^pi P_k(cos b) sin b db = (2 pi/B) delta(k,0)
    for every degree k < 2B: the quadrature is exact on H_{2B} in beta."""
    special = pytest.importorskip("scipy.special")
    w = oracle.weights(B)
    x = np.cos(oracle.beta(B))
    for k in range(0, 2 * B):
        s = float(np.sum(w * special.eval_legendre(k, x)))
        ref = 2 * math.pi / B if k == 0 else 0.0
        assert abs(s - ref) < 1e-13, (k, s)


def test_beta_grid():
    B = 5
    b = oracle.beta(B)
    assert np.allclose(b, (2 * np.arange(2 * B) + 1) * math.pi / (4 * B), rtol=0, atol=0)


@pytest.mark.parametrize("n", [1, 2, 4, 6, 8, 12, 32, 64])
def test_dft1_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(oracle.dft1(x, -1), np.fft.fft(x), atol=1e-12)
    assert np.allclose(oracle.dft1(x, +1), n * np.fft.ifft(x), atol=1e-12)


@pytest.mark.parametrize("n", [2, 6, 16])
def test_dft2_slices_matches_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n, n)) + 1j * rng.standard_normal((3, n, n))
    assert np.allclose(oracle.dft2_slices(x, -1), np.fft.fft2(x), atol=1e-11)
    assert np.allclose(oracle.dft2_slices(x, +1), n * n * np.fft.ifft2(x), atol=1e-11)
