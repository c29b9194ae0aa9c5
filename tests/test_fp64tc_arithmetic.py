"""The arithmetic the FP64-accurate tensor-core mode rests on, modelled exactly
on the host (Python integers and IEEE float32/float64 in numpy).  These check
the bounds the kernels' exactness argument uses, not the kernels themselves
(tests/test_gpu_fp64tc.py compares the kernels with the oracle):

* balanced base-128 digits: |q| <= 64, v 2^a = sum_i q_i 2^(-6-7i) to within
  2^-49 (rounding) of the scale;
* digit-level sums over K <= 1024 products stay integers below 2^24 for levels
  0..3, so FP32 accumulation of them is exact, and the level recombination in
  64-bit integers reproduces the exact dot product to the truncation bound;
* the double-float building blocks: Knuth's two-sum and the FMA-based product
  error are exact in float32, and a double-float DFT built from them matches
  the FP64 DFT to ~1e-14.
"""
import math

import numpy as np
import pytest

DIG = 7


def digits(v: float, alpha: int):
    """Balanced base-128 digits of round(v 2^(alpha+48)), as the kernel cuts them."""
    N = int(round(math.ldexp(v, alpha + 48)))  # round half to even here; the kernel rounds half up
    q = [0] * DIG
    for i in range(DIG - 1, 0, -1):
        t = N + 64
        q[i] = (t & 127) - 64
        N = t >> 7
    q[0] = N
    return q


def value(q, alpha):
    return sum(qi * 2.0 ** (-6 - 7 * i) for i, qi in enumerate(q)) * 2.0 ** (-alpha)


def test_digits_are_balanced_and_reconstruct():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        v = rng.uniform(-1.0, 1.0) * 2.0 ** rng.integers(-30, 1)
        q = digits(v, 0)
        assert all(-64 <= qi <= 64 for qi in q)
        # sum_i q_i 128^(6-i) is exactly the rounded fixed-point integer
        assert sum(qi * 128 ** (DIG - 1 - i) for i, qi in enumerate(q)) == int(round(math.ldexp(v, 48)))
        assert abs(value(q, 0) - v) <= 2.0 ** -49


def test_extreme_digits_stay_within_64():
    for v in (1.0, -1.0, 1.0 - 2.0 ** -52, -(1.0 - 2.0 ** -52), 2.0 ** -49, 0.0):
        assert all(-64 <= qi <= 64 for qi in digits(v, 0))


K7 = sum(64 * 128 ** i for i in range(DIG))


def kernel_digits(v: float, alpha: int):
    """The kernel's cut, step by step in Python integers: T = floor(v 2^(alpha+49))
    by an arithmetic shift of the signed significand, Q = T + 1 + 2 K7, and the
    digits q_i = field of Q at bit 1 + 7 (6 - i), minus 64 (digits 6..4 from the
    low 32-bit word, 3..0 from Q >> 22)."""
    b = int(np.float64(v).view(np.int64))
    e = (b >> 52) & 0x7FF
    s = min(1026 - alpha - e, 63)
    M = (b & ((1 << 52) - 1)) | (1 << 52)
    T = (-M if b < 0 else M) >> s  # Python's >> floors, like the arithmetic shift
    Q = T + 1 + 2 * K7
    assert 0 <= Q < 2 ** 51
    lo, hi = Q & 0xFFFFFFFF, (Q >> 22) & 0xFFFFFFFF
    return [(hi >> 21) - 64, ((hi >> 14) & 127) - 64, ((hi >> 7) & 127) - 64, (hi & 127) - 64,
            ((lo >> 15) & 127) - 64, ((lo >> 8) & 127) - 64, ((lo >> 1) & 127) - 64]


def balanced(N: int):
    """Balanced base-128 digits of N by the carry chain (lower six in [-64, 63])."""
    q = [0] * DIG
    for i in range(DIG - 1, 0, -1):
        t = N + 64
        q[i] = (t & 127) - 64
        N = t >> 7
    q[0] = N
    return q


def test_kernel_cut_is_balanced_digits_of_the_rounded_integer():
    """The kernel's independent bit fields give the balanced digits of
    N = floor(v 2^(alpha+48) + 1/2), over the whole range |v 2^alpha| <= 1."""
    rng = np.random.default_rng(11)
    vals = [0.0, -0.0, 1.0, -1.0, 1.0 - 2.0 ** -52, -(1.0 - 2.0 ** -52), 2.0 ** -49, -2.0 ** -49, 2.0 ** -50,
            3 * 2.0 ** -50, -3 * 2.0 ** -50, 2.0 ** -60, 5e-324]
    vals += [float(x) for x in rng.uniform(-1.0, 1.0, 5000) * 2.0 ** rng.integers(-40, 1, 5000)]
    for alpha in (0, 3, -7):
        for v0 in vals:
            v = math.ldexp(v0, -alpha)  # |v 2^alpha| <= 1
            # N = floor(v 2^(alpha+48) + 1/2) exactly, from v = +-M 2^(e-1075) (zero and subnormals: 0)
            b = int(np.float64(v).view(np.int64))
            e = (b >> 52) & 0x7FF
            M = ((b & ((1 << 52) - 1)) | (1 << 52)) * (-1 if b < 0 else 1)
            k = e - 1075 + alpha + 48
            N = 0 if e == 0 else (M << k if k >= 0 else (M + (1 << (-k - 1))) >> -k)
            q = kernel_digits(v, alpha)
            assert q == balanced(N), (v, alpha)
            assert all(-64 <= qi <= 64 for qi in q)
            assert abs(value(q, alpha) - v) <= 2.0 ** (-49 - alpha)


def test_level_sums_exact_and_recombination():
    """K = 1024 products of digit vectors: level sums 0..3 below 2^24 even with
    adversarial (all-extreme) digits, and the integer recombination equals the
    exact product of the truncated operands up to the dropped levels."""
    K = 1024
    rng = np.random.default_rng(7)
    worst = np.full((K, DIG), 64, dtype=np.int64)
    for lev in range(4):
        s = sum(int((worst[:, i] * worst[:, lev - i]).sum()) for i in range(lev + 1))
        assert abs(s) <= 2 ** 24
    a = rng.uniform(-1, 1, K) * rng.uniform(0, 1, K) ** 4  # many entries small against the scale
    x = rng.uniform(-1, 1, K)
    qa = np.array([digits(v, 0) for v in a], dtype=np.int64)
    qx = np.array([digits(v, 0) for v in x], dtype=np.int64)
    levels = [sum(int((qa[:, i] * qx[:, k - i]).sum()) for i in range(max(0, k - DIG + 1), min(k, DIG - 1) + 1))
              for k in range(DIG)]
    for k in range(4):
        assert abs(levels[k]) < 2 ** 24
    # X = 2^39 T with T = sum_k 2^-7k L_k: exact for levels 0..3, level 4..6 at 2^-39 resolution
    X = (((levels[0] * 128 + levels[1]) * 128 + levels[2]) * 128 + levels[3]) * 2 ** 18
    rest = levels[4] + levels[5] / 128 + levels[6] / 16384
    X += round(rest * 2 ** 11)
    got = X * 2.0 ** -39 * 2.0 ** -12
    exact = float(np.dot(a.astype(np.float64), x))
    scale = float(np.sum(np.abs(a) * np.abs(x)))
    assert abs(got - exact) <= 16 * K ** 0.5 * 2.0 ** -49 + 2.0 ** -45 * scale


def two_sum(a, b):
    a, b = np.float32(a), np.float32(b)
    s = np.float32(a + b)
    bb = np.float32(s - a)
    e = np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))
    return s, e


def test_two_sum_is_exact_in_float32():
    rng = np.random.default_rng(11)
    a = (rng.standard_normal(5000) * 2.0 ** rng.integers(-20, 20, 5000)).astype(np.float32)
    b = (rng.standard_normal(5000) * 2.0 ** rng.integers(-20, 20, 5000)).astype(np.float32)
    for x, y in zip(a, b):
        s, e = two_sum(x, y)
        assert float(s) + float(e) == float(x) + float(y)


def test_fma_product_error_is_exact():
    """p = fl(a b) and e = a b - p: e is a float32 (what fmaf(a, b, -p) returns)."""
    rng = np.random.default_rng(13)
    a = rng.standard_normal(5000).astype(np.float32)
    b = rng.standard_normal(5000).astype(np.float32)
    for x, y in zip(a, b):
        p = np.float32(x * y)
        e_exact = float(x) * float(y) - float(p)  # exact in float64 (48-bit product)
        assert float(np.float32(e_exact)) == e_exact


def _df_from(x):
    hi = np.float32(x)
    return hi, np.float32(x - np.float64(hi))


def _df_add(a, b):
    s, e = two_sum(a[0], b[0])
    e = np.float32(e + np.float32(a[1] + b[1]))
    s2 = np.float32(s + e)
    return s2, np.float32(e - np.float32(s2 - s))


def _df_mul(a, b):
    p = np.float32(a[0] * b[0])
    e = np.float32(float(a[0]) * float(b[0]) - float(p))  # the FMA residual
    e = np.float32(e + np.float32(a[0] * b[1]) + np.float32(a[1] * b[0]))
    s = np.float32(p + e)
    return s, np.float32(e - np.float32(s - p))


@pytest.mark.parametrize("n", [8, 32])
def test_double_float_dft_matches_fp64(n):
    """A radix-2 decimation-in-time DFT in the double-float arithmetic above,
    against numpy's FP64 FFT: the error is ~2^-47 per stage, norm-wise."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    logn = n.bit_length() - 1
    br = [int(format(i, f"0{logn}b")[::-1], 2) for i in range(n)]
    re = [_df_from(x[br[i]].real) for i in range(n)]
    im = [_df_from(x[br[i]].imag) for i in range(n)]
    size = 2
    while size <= n:
        half = size // 2
        for g in range(0, n, size):
            for k in range(half):
                c, s = math.cos(-2 * math.pi * k / size), math.sin(-2 * math.pi * k / size)
                wr, wi = _df_from(c), _df_from(s)
                i, j = g + k, g + k + half
                tr = _df_add(_df_mul(wr, re[j]), _df_mul((-wi[0], -wi[1]), im[j]))
                ti = _df_add(_df_mul(wr, im[j]), _df_mul(wi, re[j]))
                re[j] = _df_add(re[i], (-tr[0], -tr[1]))
                im[j] = _df_add(im[i], (-ti[0], -ti[1]))
                re[i] = _df_add(re[i], tr)
                im[i] = _df_add(im[i], ti)
        size *= 2
    got = np.array([float(r[0]) + float(r[1]) + 1j * (float(q[0]) + float(q[1])) for r, q in zip(re, im)])
    ref = np.fft.fft(x)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert 0 < err < 1e-13, err  # nonzero: the double-float rounding is visible against FP64
