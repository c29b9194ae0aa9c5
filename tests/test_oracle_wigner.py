"""Pins for the oracle's Wigner-d functions (Sec. 2.2 of the paper).

Each test checks the oracle against something other than itself: closed forms
worked out by hand from the explicit Jacobi form, sympy's Wigner-d (a textbook
routine; the paper's d(l,m,m') is the transpose of the d^l_{m m'} of sympy /
Sakurai), scipy's Jacobi polynomials, high-precision mpmath evaluations, the
symmetries of Eq. (Wigner_symmetries) and orthogonality under the quadrature.
"""
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1808)


def d1_table(b):
    """d(1,m,m';b), rows m = -1,0,1, columns m' = -1,0,1 (paper's convention)."""
    c2, s2, r = math.cos(b / 2) ** 2, math.sin(b / 2) ** 2, math.sin(b) / math.sqrt(2)
    return np.array([[c2, -r, s2],
                     [r, math.cos(b), -r],
                     [s2, r, c2]])


D2_CLOSED = {
    (0, 0): lambda b: 1 - 1.5 * math.sin(b) ** 2,
    (0, 1): lambda b: -math.sqrt(6) / 4 * math.sin(2 * b),
    (1, 0): lambda b: math.sqrt(6) / 4 * math.sin(2 * b),
    (1, 1): lambda b: math.cos(b / 2) * math.cos(3 * b / 2),
    (2, 2): lambda b: math.cos(b / 2) ** 4,
    (2, -2): lambda b: math.sin(b / 2) ** 4,
    (-2, -1): lambda b: -(1 + math.cos(b)) * math.sin(b) / 2,
    (0, 2): lambda b: math.sqrt(6) / 4 * math.sin(b) ** 2,
}


@pytest.mark.parametrize("b", list(RNG.uniform(0.01, math.pi - 0.01, size=20)))
def test_d1_closed_form(b):
    tab = d1_table(b)
    for a, m in enumerate((-1, 0, 1)):
        for c, mp in enumerate((-1, 0, 1)):
            assert abs(oracle.wigner_d_explicit(1, m, mp, b) - tab[a, c]) < 1e-15
            col = oracle.wigner_d_column(2, m, mp, b)  # l = max(|m|,|m'|)..1
            assert abs(col[1 - max(abs(m), abs(mp))] - tab[a, c]) < 1e-15


@pytest.mark.parametrize("b", list(RNG.uniform(0.01, math.pi - 0.01, size=20)))
def test_d2_closed_form(b):
    for (m, mp), f in D2_CLOSED.items():
        assert abs(oracle.wigner_d_explicit(2, m, mp, b) - f(b)) < 1e-15
        col = oracle.wigner_d_column(3, m, mp, b)
        assert abs(col[2 - max(abs(m), abs(mp))] - f(b)) < 1e-15


def test_matches_sympy_transposed():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.quantum.spin import Rotation

    b = 0.8371
    for l in range(0, 4):
        for m in range(-l, l + 1):
            for mp in range(-l, l + 1):
                ref = complex(sympy.N(Rotation.d(l, mp, m, b).doit(), 30))
                assert abs(ref.imag) < 1e-14
                assert abs(oracle.wigner_d_explicit(l, m, mp, b) - ref.real) < 1e-14, (l, m, mp)
                col = oracle.wigner_d_column(l + 1, m, mp, b)
                assert abs(col[l - max(abs(m), abs(mp))] - ref.real) < 1e-14, (l, m, mp)


def test_jacobi_matches_scipy():
    special = pytest.importorskip("scipy.special")
    for n in range(0, 12):
        for a in range(0, 6):
            for bb in range(0, 6):
                for x in (-0.93, -0.2, 0.31, 0.77):
                    ref = special.eval_jacobi(n, a, bb, x)
                    # the explicit alternating sum cancels (terms up to ~1e7 here), so a few
                    # digits go; any wrong index or sign would be off by O(1)
                    assert abs(oracle.jacobi(n, a, bb, x) - ref) <= 1e-10 * max(1.0, abs(ref))


def test_recurrence_matches_explicit_all_orders():
    """Eq. (Wigner_d_recurrence) from the seeds vs the explicit form, l < 16."""
    B = 16
    for b in (0.05, 0.9, 1.6, 2.7, 3.1):
        for m in range(1 - B, B):
            for mp in range(1 - B, B):
                col = oracle.wigner_d_column(B, m, mp, b)
                l0 = max(abs(m), abs(mp))
                ref = np.array([oracle.wigner_d_explicit(l, m, mp, b) for l in range(l0, B)])
                # the explicit alternating sum loses digits as l grows (1e-11 at l = 23,
                # where the recurrence still matches 50-digit values); larger l is
                # pinned in test_recurrence_large_degree_high_precision
                assert np.max(np.abs(col - ref)) < 1e-12, (m, mp, b)


def test_symmetries_of_recurrence():
    """The seven relations of Eq. (Wigner_symmetries), on recurrence columns, l < 31."""
    B = 31
    for b in RNG.uniform(0.05, math.pi - 0.05, size=4):
        for m in range(0, B):
            for mp in range(-m, m + 1):
                l0 = max(abs(m), abs(mp))
                ls = np.arange(l0, B)
                d = oracle.wigner_d_column(B, m, mp, b)
                pm = (-1.0) ** (m - mp)
                sl_mp = (-1.0) ** (ls - mp)
                sl_m = (-1.0) ** (ls + m)
                rel = [
                    (pm, oracle.wigner_d_column(B, -m, -mp, b)),
                    (pm, oracle.wigner_d_column(B, mp, m, b)),
                    (sl_mp, oracle.wigner_d_column(B, -m, mp, math.pi - b)),
                    (sl_m, oracle.wigner_d_column(B, m, -mp, math.pi - b)),
                    (sl_mp, oracle.wigner_d_column(B, -mp, m, math.pi - b)),
                    (sl_m, oracle.wigner_d_column(B, mp, -m, math.pi - b)),
                    (1.0, oracle.wigner_d_column(B, -mp, -m, b)),
                ]
                for s, other in rel:
                    assert np.max(np.abs(d - s * other)) < 1e-13, (m, mp)


def test_seed_log_domain_high_precision():
    """Seeds at large orders, where factorials overflow FP64, vs 40-digit mpmath."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    cases = [(500, 3), (500, -499), (-511, 200), (37, 511), (3, -510), (511, 511), (400, 0)]
    for m, mp in cases:
        for b in (0.1, 0.7, 1.5, 2.9):
            bb = mpmath.mpf(b)
            c, s = mpmath.cos(bb / 2), mpmath.sin(bb / 2)
            if abs(m) >= abs(mp):
                mu = abs(m)
                if m >= 0:
                    val = mpmath.sqrt(mpmath.binomial(2 * mu, mu + mp)) * c ** (mu + mp) * s ** (mu - mp)
                else:
                    val = mpmath.sqrt(mpmath.binomial(2 * mu, mu + mp)) * c ** (mu - mp) * (-s) ** (mu + mp)
            else:
                mu = abs(mp)
                if mp >= 0:
                    val = mpmath.sqrt(mpmath.binomial(2 * mu, mu + m)) * c ** (mu + m) * (-s) ** (mu - m)
                else:
                    val = mpmath.sqrt(mpmath.binomial(2 * mu, mu + m)) * c ** (mu - m) * s ** (mu + m)
            ref = float(val)
            got = oracle.wigner_seed(m, mp, b)
            if abs(ref) < 1e-300:
                assert abs(got) < 1e-290
            else:
                assert abs(got - ref) <= 1e-12 * abs(ref), (m, mp, b, got, ref)


def test_recurrence_large_degree_high_precision():
    """Recurrence values at l up to 511 vs the explicit form summed in 60-digit mpmath."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    B = 512
    for m, mp in [(0, 0), (5, -2), (100, 37), (-300, 12), (12, 450)]:
        for b in (0.3, 1.9):
            col = oracle.wigner_d_column(B, m, mp, b)
            l0 = max(abs(m), abs(mp))
            for l in (l0 + 1, (l0 + B) // 2, B - 1):
                # explicit form, reduced to m' >= |m| by the beta-preserving symmetries
                mm, nn, sg = m, mp, 1
                if abs(nn) >= abs(mm):
                    if nn < 0:
                        mm, nn, sg = -mm, -nn, (-1) ** (m - mp)
                else:
                    if mm >= 0:
                        mm, nn, sg = nn, mm, (-1) ** (m - mp)
                    else:
                        mm, nn, sg = -nn, -mm, 1
                bb = mpmath.mpf(b)
                fac = mpmath.sqrt(mpmath.factorial(l + nn) * mpmath.factorial(l - nn)
                                  / (mpmath.factorial(l + mm) * mpmath.factorial(l - mm)))
                val = ((-1) ** (mm + nn) * fac * mpmath.sin(bb / 2) ** (nn - mm)
                       * mpmath.cos(bb / 2) ** (mm + nn)
                       * mpmath.jacobi(l - nn, nn - mm, mm + nn, mpmath.cos(bb)))
                ref = sg * float(val)
                got = col[l - l0]
                assert abs(got - ref) < 1e-12, (m, mp, l, b, got, ref)


def _orth_err(B, pairs):
    w = oracle.weights(B)
    bj = oracle.beta(B)
    worst = 0.0
    for m, mp in pairs:
        l0 = max(abs(m), abs(mp))
        T = np.stack([oracle.wigner_d_column(B, m, mp, x) for x in bj], axis=1)  # [l][j]
        G = (B / math.pi) * (T * w[None, :]) @ T.T
        ls = np.arange(l0, B)
        worst = max(worst, float(np.max(np.abs(G - np.diag(2.0 / (2 * ls + 1))))))
    return worst


@pytest.mark.parametrize("B", [1, 2, 5, 8, 16])
def test_orthogonality_under_quadrature_all_orders(B):
    """(B/pi) sum_j w_B(j) d(l,m,m';b_j) d(l',m,m';b_j) = 2/(2l+1) delta(l,l'),
    from the orthogonality relation with the exact quadrature of Eq. (quadrature)."""
    pairs = [(m, mp) for m in range(1 - B, B) for mp in range(1 - B, B)]
    assert _orth_err(B, pairs) < 1e-13


@pytest.mark.parametrize("B", [64, 512])
def test_orthogonality_under_quadrature_sampled(B):
    rng = np.random.default_rng(B)
    pairs = [(0, 0), (B - 1, B - 1), (B - 1, 1 - B), (1 - B, 0), (B // 2, -(B // 3))]
    pairs += [tuple(int(v) for v in rng.integers(1 - B, B, size=2)) for _ in range(8)]
    assert _orth_err(B, pairs) < 1e-12
