"""Pins for the oracle's whole transforms (Sec. 2.3-2.4 of the paper).

* fast (separation of variables + DWT) = the direct O(B^6) sums of
  Eq. (quadrature) / Eq. (fourier_representation), on any grid
* one-hot: a single Wigner-D function sampled on the grid (built here from
  scipy's Jacobi polynomials, not from the oracle) maps to one coefficient
* forward(inverse(c)) = c on H_B (sampling theorem), Parseval, real-input
  conjugate symmetry, the layout of the coefficient array
"""
import math

import numpy as np
import pytest

import oracle
from paper_1808_00896_gb300 import synth


def test_num_coeffs_and_layout():
    for B in (1, 2, 3, 7, 16):
        assert oracle.num_coeffs(B) == B * (4 * B * B - 1) // 3
        lmm = oracle.coef_lmm(B)
        assert len(lmm) == oracle.num_coeffs(B)
        assert np.array_equal(lmm[:, 0], synth.coef_degrees(B))
        # each (l, m, m') with |m|,|m'| <= l < B appears exactly once
        assert len({tuple(r) for r in lmm}) == len(lmm)
        for t in range(0, len(lmm), max(1, len(lmm) // 50)):
            l, m, mp = lmm[t]
            assert oracle.coef_index(B, int(l), int(m), int(mp)) == t
    assert oracle.coef_index(4, 2, 3, 0) == -1
    assert oracle.coef_index(4, 4, 0, 0) == -1


@pytest.mark.parametrize("B", [1, 2, 3, 4, 5])
def test_fast_inverse_equals_direct(B):
    c = synth.coefficients(B, "uniform", seed=100 + B)
    assert synth.rel_l2(oracle.inverse(B, c), oracle.direct_inverse(B, c)) < 1e-14


@pytest.mark.parametrize("B", [1, 2, 3, 4, 5])
def test_fast_forward_equals_direct_any_grid(B):
    g = synth.random_grid(B, seed=200 + B)  # not band-limited: both compute the same quadrature sum
    assert synth.rel_l2(oracle.forward(B, g), oracle.direct_forward(B, g)) < 1e-14


def _wigner_D_grid(B, l, m, mp):
    """D(l,m,m') on the (2B)^3 grid from Eq. (Wigner_D), with d from the explicit
    Jacobi form via scipy (independent of the oracle); needs m' >= |m|."""
    special = pytest.importorskip("scipy.special")
    assert mp >= abs(m)
    n = 2 * B
    beta = (2 * np.arange(n) + 1) * math.pi / (4 * B)
    ang = np.arange(n) * math.pi / B
    fac = math.sqrt(math.factorial(l + mp) * math.factorial(l - mp)
                    / (math.factorial(l + m) * math.factorial(l - m)))
    d = ((-1) ** (m + mp) * fac * np.sin(beta / 2) ** (mp - m) * np.cos(beta / 2) ** (m + mp)
         * special.eval_jacobi(l - mp, mp - m, m + mp, np.cos(beta)))
    ea = np.exp(-1j * m * ang)
    eg = np.exp(-1j * mp * ang)
    return d[:, None, None] * ea[None, :, None] * eg[None, None, :]


@pytest.mark.parametrize("B,l,m,mp", [(4, 0, 0, 0), (4, 3, -2, 3), (8, 5, 1, 4), (8, 7, -7, 7),
                                      (16, 9, 3, 6), (16, 15, 0, 15)])
def test_one_hot(B, l, m, mp):
    f = oracle.forward(B, _wigner_D_grid(B, l, m, mp))
    e = np.zeros_like(f)
    e[oracle.coef_index(B, l, m, mp)] = 1.0
    assert np.max(np.abs(f - e)) < 1e-13


def test_constant_function():
    B = 8
    f = oracle.forward(B, np.ones((2 * B,) * 3))
    e = np.zeros_like(f)
    e[oracle.coef_index(B, 0, 0, 0)] = 1.0
    assert np.max(np.abs(f - e)) < 1e-14


@pytest.mark.parametrize("B,kind", [(1, "uniform"), (7, "uniform"), (16, "uniform"), (32, "gauss_decay")])
def test_round_trip(B, kind):
    c = synth.coefficients(B, kind, seed=300 + B)
    assert synth.rel_l2(oracle.forward(B, oracle.inverse(B, c)), c) < 1e-13


@pytest.mark.parametrize("B", [4, 12])
def test_parseval(B):
    """(pi/B) sum_{ijk} w_B(j)|f|^2 = sum 8 pi^2/(2l+1) |f(l,m,m')|^2: the
    orthogonality relation with the quadrature, exact for |f|^2 of bandwidth 2B-1."""
    c = synth.coefficients(B, "uniform", seed=400 + B)
    g = oracle.inverse(B, c)
    w = oracle.weights(B)
    lhs = math.pi / B * float(np.sum(w[:, None, None] * np.abs(g) ** 2))
    ls = synth.coef_degrees(B)
    rhs = float(np.sum(8 * math.pi ** 2 / (2 * ls + 1) * np.abs(c) ** 2))
    assert abs(lhs - rhs) < 1e-12 * rhs


def test_real_input_symmetry():
    """f real => f(l,-m,-m') = (-1)^(m-m') conj f(l,m,m'), from Eq. (Wigner_symmetries)."""
    B = 8
    g = synth.random_grid(B, seed=5).real.astype(np.complex128)
    f = oracle.forward(B, g)
    for l, m, mp in oracle.coef_lmm(B)[::7]:
        a = f[oracle.coef_index(B, int(l), int(m), int(mp))]
        b = f[oracle.coef_index(B, int(l), int(-m), int(-mp))]
        assert abs(a - (-1) ** int(m - mp) * np.conj(b)) < 1e-14


def test_sampled_forms_agree_with_full():
    B = 12
    g = synth.random_grid(B, seed=7)
    f = oracle.forward(B, g)
    pairs = [(0, 0), (11, -11), (-3, 7), (5, 5), (-11, 0)]
    for (m, mp), run in zip(pairs, oracle.forward_pairs(B, g, pairs)):
        l0 = max(abs(m), abs(mp))
        o = oracle.coef_index(B, l0, m, mp)
        assert np.max(np.abs(run - f[o:o + B - l0])) < 1e-13
    c = synth.coefficients(B, "gauss_decay", seed=8)
    grid = oracle.inverse(B, c)
    pts = [(0, 0, 0), (3, 23, 5), (23, 11, 17)]
    vals = oracle.inverse_points(B, c, pts)
    for (i, j, k), v in zip(pts, vals):
        assert abs(v - grid[j, i, k]) < 1e-12


def test_golden_forward_B4():
    """Regression fixture written by tests/golden/make_golden.py (direct sum)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "forward_B4_random_grid.txt")
    rows = np.loadtxt(path)
    B = 4
    g = synth.random_grid(B, seed=0x5F3F1808 + 1)
    f = oracle.forward(B, g)
    assert np.array_equal(rows[:, :3].astype(np.int64), oracle.coef_lmm(B))
    ref = rows[:, 3] + 1j * rows[:, 4]
    assert synth.rel_l2(f, ref) < 1e-14


@pytest.mark.parametrize("B", [1, 3, 6])
def test_adjoints_dot_test(B):
    """<F x, y> = <x, F^H y> and <G c, x> = <c, G^H x> with the pinned forward F
    and inverse G: a wrong term, sign or index in an adjoint breaks the identity."""
    rng = np.random.default_rng(B)
    x = synth.random_grid(B, seed=50 + B)
    y = synth.coefficients(B, "uniform", seed=60 + B)
    lhs = np.vdot(oracle.forward(B, x), y)
    rhs = np.vdot(x, oracle.forward_adjoint(B, y))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    lhs = np.vdot(oracle.inverse(B, y), x)
    rhs = np.vdot(y, oracle.inverse_adjoint(B, x))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    assert rng is not None


def test_adjoint_of_forward_is_dense_transpose():
    """Brute force on B = 2: build the forward's matrix column by column and
    compare its conjugate transpose with the adjoint applied to unit vectors."""
    B = 2
    n = 2 * B
    N = n ** 3
    M = np.zeros((oracle.num_coeffs(B), N), dtype=np.complex128)
    for t in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[t] = 1.0
        M[:, t] = oracle.forward(B, e.reshape(n, n, n))
    for t in range(oracle.num_coeffs(B)):
        e = np.zeros(oracle.num_coeffs(B), dtype=np.complex128)
        e[t] = 1.0
        assert np.allclose(oracle.forward_adjoint(B, e).reshape(-1), M.conj().T[:, t], atol=1e-14)
