"""Host models of two kernels' index arithmetic and algebra, run on the CPU.
They mirror the loops of the CUDA code (tests/test_gpu_*.py compare the kernels
themselves with the oracle):

* the FP64 slice FFT (csrc/fft_fp64.cu): bit-reversed input with the first two
  radix-2 stages fused into the load, then pairs of decimation-in-time stages
  and a last radix-2 stage, each butterfly in Goedecker's factored form
  a +- w b with w = m (1 + i tau) or i m (1 + i tau), |tau| <= 1; rows pass
  and padded columns pass, every index bounds-checked;
* the forward FP64 DWT's contraction lanes (csrc/dwt_fp64.cu): for every tile
  shape and partner count, every output column of every degree receives every
  beta sample exactly once, the combining shuffles stay inside a warp, and one
  lane writes each output.
"""
import math
from collections import Counter

import numpy as np
import pytest


# ---------------------------------------------------------------------------
# FP64 FFT
# ---------------------------------------------------------------------------
def _brev(t, bits):
    return int(format(t, f"0{bits}b")[::-1], 2) if bits else 0


def _twiddles(n, sign):
    """exp(sign 2 pi i t / n), t < n/2, as (tau, m1, m2, swap)."""
    out = []
    for t in range(n // 2):
        c, s = math.cos(2 * math.pi * t / n), sign * math.sin(2 * math.pi * t / n)
        out.append((s / c, c, c, 0) if abs(c) >= abs(s) else (-c / s, -s, s, 1))
    return out


def _bfly(a, b, w):
    tau, m1, m2, swap = w
    zr, zi = b.real - tau * b.imag, b.imag + tau * b.real
    p, q = (zi, zr) if swap else (zr, zi)
    return complex(a.real + m1 * p, a.imag + m2 * q), complex(a.real - m1 * p, a.imag - m2 * q)


def _first_radix4(x0, x1, x2, x3, conj):
    a0, a1, a2, a3 = x0 + x1, x0 - x1, x2 + x3, x2 - x3
    u, v = a1 + 1j * a3, a1 - 1j * a3
    return [a0 + a2, v if conj else u, a0 - a2, u if conj else v]


def _stages(s, cnt, ld, n, logn, h, lh, tw):
    while 4 * h <= n:
        for q in range(cnt * (n >> 2)):
            row, qq = q >> (logn - 2), q & ((n >> 2) - 1)
            k, g = qq & (h - 1), qq >> lh
            base = row * ld + g * 4 * h + k
            idx = [base, base + h, base + 2 * h, base + 3 * h]
            assert all(0 <= i - row * ld < n for i in idx)
            x = [s[i] for i in idx]
            i1, i2, i3 = k << (logn - 1 - lh), k << (logn - 2 - lh), (k + h) << (logn - 2 - lh)
            assert max(i1, i2, i3) < n // 2
            x[0], x[1] = _bfly(x[0], x[1], tw[i1])
            x[2], x[3] = _bfly(x[2], x[3], tw[i1])
            x[0], x[2] = _bfly(x[0], x[2], tw[i2])
            x[1], x[3] = _bfly(x[1], x[3], tw[i3])
            for i, v in zip(idx, x):
                s[i] = v
        h, lh = 4 * h, lh + 2
    if 2 * h == n:
        for b in range(cnt * h):
            row, k = b >> lh, b & (h - 1)
            i = row * ld + k
            s[i], s[i + h] = _bfly(s[i], s[i + h], tw[k])


def _dft_rows(x, sign):
    """The rows pass on a (rows, n) array, one block of rows at a time."""
    rows_total, n = x.shape
    logn, conj, tw = n.bit_length() - 1, sign < 0, _twiddles(n, sign)
    out = np.empty_like(x)
    for r in range(rows_total):
        s = [0j] * n
        if logn >= 2:
            n4 = n >> 2
            for t in range(n4):
                d = 4 * _brev(t, logn - 2)
                s[d:d + 4] = _first_radix4(x[r, t], x[r, t + n // 2], x[r, t + n4], x[r, t + 3 * n4], conj)
            _stages(s, 1, n, n, logn, 4, 2, tw)
        else:
            s = list(x[r])
            _stages(s, 1, n, n, logn, 1, 0, tw)
        out[r] = s
    return out


def _dft_columns(x, sign):
    """The columns pass on one n x n slice: kb columns per block, column c of
    the block at s + c (n + 1)."""
    n = x.shape[0]
    logn, conj, tw = n.bit_length() - 1, sign < 0, _twiddles(n, sign)
    kb, ld = min(n, max(2, 1024 // n)), n + 1
    out = x.copy()
    for k0 in range(0, n, kb):
        s = [0j] * (kb * ld)
        if logn >= 2:
            n4 = n >> 2
            for q in range(kb * n4):
                t, c = q // kb, q % kb
                col = x[:, k0 + c]
                d = c * ld + 4 * _brev(t, logn - 2)
                s[d:d + 4] = _first_radix4(col[t], col[t + n // 2], col[t + n4], col[t + 3 * n4], conj)
            _stages(s, kb, ld, n, logn, 4, 2, tw)
        else:
            for e in range(kb * n):
                i, c = e // kb, e % kb
                s[c * ld + i] = x[i, k0 + c]
            _stages(s, kb, ld, n, logn, 1, 0, tw)
        for e in range(kb * n):
            i, c = e // kb, e % kb
            out[i, k0 + c] = s[c * ld + i]
    return out


def test_twiddle_factorisation():
    """Both factored forms reproduce exp(i theta) with |tau| <= 1."""
    for n in (2, 8, 128, 1024):
        for sign in (1, -1):
            for t, (tau, m1, m2, swap) in enumerate(_twiddles(n, sign)):
                assert abs(tau) <= 1.0
                w = complex(m1, m1 * tau) if not swap else 1j * m2 * complex(1.0, tau)
                assert abs(w - np.exp(sign * 2j * np.pi * t / n)) < 1e-15


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128, 1024])
@pytest.mark.parametrize("sign", [1, -1])
def test_fft_rows_model_matches_numpy(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    ref = np.fft.ifft(x, axis=1) * n if sign > 0 else np.fft.fft(x, axis=1)
    assert np.linalg.norm(_dft_rows(x, sign) - ref) <= 2e-15 * max(1, math.log2(n)) * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [2, 4, 8, 32, 64])
@pytest.mark.parametrize("sign", [1, -1])
def test_fft_2d_model_matches_numpy(n, sign):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    got = _dft_columns(_dft_rows(x, sign), sign)
    ref = np.fft.ifft2(x) * n * n if sign > 0 else np.fft.fft2(x)
    assert np.linalg.norm(got - ref) <= 4e-15 * max(1, math.log2(n)) * np.linalg.norm(ref)


# ---------------------------------------------------------------------------
# Forward FP64 DWT: contraction lanes
# ---------------------------------------------------------------------------
def _lane_map(NT, TPI, n, npc, nt):
    """Mirror of the forward kernel's phase-B mapping for one degree tile of
    nt degrees and npc contracted partners."""
    LT = NT // (16 * TPI)
    cover, writers, lanes = Counter(), Counter(), {}
    fold = TPI <= 2 and npc <= 4
    for tid in range(NT):
        half, ot = tid % TPI, tid // TPI
        pt, pc = ot >> 4, (ot & 7) if fold else (ot & 15)
        upper = (ot >> 3) & 1 if fold else 0
        parts = 2 * TPI if fold else TPI
        part = half + TPI * upper
        jlen = (n + parts - 1) // parts
        jbeg = min(n, part * jlen)
        jcnt = min(jlen, n - jbeg)
        active = pt < nt and (pc >> 1) < npc
        assert pt < LT
        if active:
            for j in range(jbeg, jbeg + jcnt):
                cover[(pt, pc, j)] += 1
            if half == 0 and upper == 0:
                writers[(pt, pc)] += 1
        lanes[tid] = (pt, pc, active)
    masks = ([1] if TPI >= 2 else []) + ([2] if TPI >= 4 else []) + ([8 * TPI] if fold else [])
    return cover, writers, lanes, masks


@pytest.mark.parametrize("NT,TPI", [(256, 1), (256, 2), (128, 1), (512, 4), (256, 4)])
@pytest.mark.parametrize("n", [2, 6, 10, 64, 130, 258, 514])
@pytest.mark.parametrize("npc", [1, 2, 4, 8])
def test_forward_lane_mapping(NT, TPI, n, npc):
    LT = NT // (16 * TPI)
    for nt in sorted({1, LT}):
        cover, writers, lanes, masks = _lane_map(NT, TPI, n, npc, nt)
        for tid in range(NT):
            for mk in masks:
                o = tid ^ mk
                assert o // 32 == tid // 32, "a shuffle leaves the warp"
                a, b = lanes[tid], lanes[o]
                if a[2] or b[2]:
                    assert a[:2] == b[:2], "a shuffle combines different outputs"
        for pt in range(nt):
            for pc in range(2 * npc):
                assert writers[(pt, pc)] == 1
                assert all(cover[(pt, pc, j)] == 1 for j in range(n))
        assert all(v == 1 for v in cover.values())


# ---------------------------------------------------------------------------
# Mixed-precision forward DWT pipeline (dwt_mixed.cu, dwt_forward_mixed_kernel):
# step `it` waits for chunk it-1's MMA, folds the accumulator into the
# compensated sums at the end of each drain group of G chunks (the tile's
# first group starts them; a tile of one group keeps its accumulator), finishes
# the tile after its last chunk, then refills the one operand stage with chunk
# it and issues its MMA (accumulating unless it starts a group).  A host model
# of that schedule with the accumulator's contents tracked: the stage is never
# refilled while an MMA that reads it may still run, every chunk's product
# reaches the tile's result exactly once, and every tile gets one epilogue.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,n", [(1, 2), (5, 16), (64, 128), (65, 128), (130, 256), (512, 1024), (200, 1024)])
@pytest.mark.parametrize("KC", [128, 256])
@pytest.mark.parametrize("G", [1, 4])
def test_mixed_forward_pipeline_schedule(L, n, KC, G):
    TM = 64
    nch = -(-n // KC)
    ntiles = -(-L // TM)
    total = ntiles * nch
    comp = nch > G
    pending = None   # chunk whose MMA reads the stage and has not been waited for
    acc = []         # chunks summed in the TMEM accumulator
    sums = None      # chunks in the compensated (hi, lo) sums
    results = {}
    for it in range(total + 1):
        if it > 0:
            prev = it - 1
            assert pending == prev  # wait for chunk it-1's MMA
            pending = None
            pc = prev % nch
            if comp and (pc % G == G - 1 or pc == nch - 1):
                sums = list(acc) if pc < G else sums + acc   # first drain of the tile starts the sums
            if pc == nch - 1:
                results[prev // nch] = sums if comp else list(acc)
        if it < total:
            assert pending is None  # the stage's last reader has completed
            c = it % nch
            acc = [it] if c % G == 0 else acc + [it]   # a group starts a fresh accumulator
            pending = it
    assert pending is None
    assert sorted(results) == list(range(ntiles))
    for t, chunks in results.items():
        assert sorted(chunks) == list(range(t * nch, (t + 1) * nch)), (t, chunks)


# ---------------------------------------------------------------------------
# Real-grid slice FFT (fft_fp64.cu, fft64_rows_r2c_kernel / _c2r_kernel): the
# unpacking identities of the half-length complex DFT, modelled in numpy and
# checked against the direct DFT (exp(s 2 pi i k t / n), unnormalised).
# ---------------------------------------------------------------------------
def _dft(x, s):
    n = len(x)
    k = np.arange(n)
    return np.exp(s * 2j * np.pi * np.outer(k, k) / n) @ x


@pytest.mark.parametrize("n", [2, 4, 8, 16, 64])
@pytest.mark.parametrize("s", [1, -1])
def test_real_row_r2c_unpacking(n, s):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    N = n // 2
    Z = _dft(x[0::2] + 1j * x[1::2], s)          # the N-point DFT of the packed samples
    k = np.arange(N)
    b = Z[(N - k) % N]
    E = 0.5 * (Z + np.conj(b))
    O = (Z - np.conj(b)) / 2j
    X = E + np.exp(s * 2j * np.pi * k / n) * O
    assert np.allclose(X, _dft(x, s)[:N], rtol=0, atol=1e-12 * n)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 64])
@pytest.mark.parametrize("s", [1, -1])
def test_real_row_c2r_packing(n, s):
    rng = np.random.default_rng(100 + n)
    N = n // 2
    X = np.zeros(n, dtype=complex)
    X[0] = rng.standard_normal()
    X[1:N] = rng.standard_normal(N - 1) + 1j * rng.standard_normal(N - 1)
    X[N + 1:] = np.conj(X[1:N][::-1])             # Hermitian, Nyquist term 0
    want = _dft(X, s)
    assert np.abs(want.imag).max() < 1e-12 * n
    k = np.arange(N)
    b = np.where(k > 0, X[(N - k) % n], 0)        # X[N - k], with X[N] = 0
    Z = (X[:N] + np.conj(b)) + 1j * np.exp(s * 2j * np.pi * k / n) * (X[:N] - np.conj(b))
    z = _dft(Z, s)
    x = np.empty(n)
    x[0::2], x[1::2] = z.real, z.imag
    assert np.allclose(x, want.real, rtol=0, atol=1e-12 * n)
