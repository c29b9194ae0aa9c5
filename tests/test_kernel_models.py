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
  lane writes each output;
* the real-grid form of the double-float slice FFT (csrc/fft_df.cu): the
  blocks, bit-reversed slots, power-of-two scales and unpacking / packing of
  fft_rows_r2c_kernel, fft_cols_kernel on m' < B, fft_cols_f64_kernel and
  fft_rows_c2r_kernel, in complex128, against numpy.fft on whole grids, with
  every index bounds-checked and the launch shapes checked for B = 2..512.
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



# ---------------------------------------------------------------------------
# Real-grid double-float slice FFT (fft_df.cu): the kernels' loops over blocks,
# bit-reversed slots and scales, in complex128.  Launch shapes as the host
# code computes them: n = 2B, N = B; r2c rows rpb = min(256, max(1, 1024 / N)),
# c2r rows rpb = min(n, max(1, 1024 / N)), columns kb = min(N, max(4, 4096 / n)).
# ---------------------------------------------------------------------------
ZERO_ROW = -100000


def _df_shapes(B):
    n, N = 2 * B, B
    return (n, N, min(256, max(1, 1024 // N)), min(n, max(1, 1024 // N)), min(N, max(4, 4096 // n)))


def _df_stages(s, cnt, n, logn, tw, conj):
    """dft_stages of fft_df.cu: radix-4 passes (sub-stages 2h and 4h), then a
    last radix-2 stage when log2 n is odd; tw[t] = exp(+2 pi i t / n)."""
    T = np.conj(tw) if conj else tw
    h, lh = 1, 0
    while 4 * h <= n:
        for q in range(cnt * (n >> 2)):
            row, qq = q >> (logn - 2), q & ((n >> 2) - 1)
            k, g = qq & (h - 1), qq >> lh
            i0 = row * n + g * 4 * h + k
            assert i0 + 3 * h < cnt * n and (k << (logn - 1 - lh)) < len(T)
            w1, w2 = T[k << (logn - 1 - lh)], T[k << (logn - 2 - lh)]
            x0, x1, x2, x3 = s[i0], s[i0 + h], s[i0 + 2 * h], s[i0 + 3 * h]
            t1, t3 = w1 * x1, w1 * x3
            a0, a1, a2, a3 = x0 + t1, x0 - t1, x2 + t3, x2 - t3
            u2, u3 = w2 * a2, (w2 * a3) * (-1j if conj else 1j)
            s[i0], s[i0 + 2 * h], s[i0 + h], s[i0 + 3 * h] = a0 + u2, a0 - u2, a1 + u3, a1 - u3
        h, lh = 4 * h, lh + 2
    if 2 * h == n:
        for b in range(cnt * (n >> 1)):
            row, k = b >> (logn - 1), b & (h - 1)
            i, j = row * n + k, row * n + k + h
            t = T[k] * s[j]
            s[i], s[j] = s[i] + t, s[i] - t


def _exp_of(v):
    """Biased FP64 exponent of the larger part (0 for zero), as the kernels read it."""
    m = max(abs(v.real), abs(v.imag))
    return 0 if m == 0 else math.frexp(m)[1] - 1 + 1023


def _df_r2c(B, x, sign):
    """fft_rows_r2c_kernel, then fft_cols_kernel on the columns m' < B; returns
    S (n, n, n) with the columns >= B left NaN, and the row scales."""
    n, N, rpb, _, kb = _df_shapes(B)
    logn, logN, conj = n.bit_length() - 1, N.bit_length() - 1, sign < 0
    tw = np.exp(2j * np.pi * np.arange(n // 2) / n)
    twN = tw[0:2 * (N >> 1):2]
    z = x.reshape(-1)[0::2] + 1j * x.reshape(-1)[1::2]
    work = np.full(n ** 3, np.nan + 0j)
    rexp = np.full(n * n, 7777)
    nrows = n * n
    written = np.zeros(n ** 3, dtype=int)
    for blk in range((nrows + rpb - 1) // rpb):
        r0 = blk * rpb
        rows = min(rpb, nrows - r0)
        assert rows <= 256
        sm = np.full(rpb * N, np.nan + 0j)
        rmax = [0] * rows
        for e in range(rows * N):
            assert r0 * N + e < len(z)
            rmax[e >> logN] = max(rmax[e >> logN], _exp_of(z[r0 * N + e]))
            sm[(e >> logN) * N + _brev(e & (N - 1), logN)] = z[r0 * N + e]
        for e in range(rows * N):
            rl = e >> logN
            i = rl * N + _brev(e & (N - 1), logN)
            sm[i] *= 2.0 ** ((1023 - rmax[rl]) if rmax[rl] else 0)
        for t in range(rows):
            rexp[r0 + t] = rmax[t] - 1023 if rmax[t] else ZERO_ROW
        _df_stages(sm, rows, N, logN, twN, conj)
        for e in range(rows * N):
            rl, k = e >> logN, e & (N - 1)
            a, b = sm[rl * N + k], sm[rl * N + ((N - k) & (N - 1))]
            E = complex(0.5 * (a.real + b.real), 0.5 * (a.imag - b.imag))
            O = complex(0.5 * (a.imag + b.imag), 0.5 * (b.real - a.real))
            o = (r0 + rl) * n + k
            assert k < N and o < n ** 3
            work[o] = E + (np.conj(tw[k]) if conj else tw[k]) * O
            written[o] += 1
    S = np.full(n ** 3, np.nan + 0j)
    tiles = N // kb
    assert tiles * kb == N and kb <= 64
    for blk in range(n * tiles):
        js, k0 = blk // tiles, (blk % tiles) * kb
        base = js * n * n + k0
        sref = max(rexp[js * n + i] for i in range(n))
        sm = np.full(kb * n, np.nan + 0j)
        for e in range(n * kb):
            i, c = e // kb, e % kb
            f = 0.0 if rexp[js * n + i] - sref < -126 else 2.0 ** (rexp[js * n + i] - sref)
            sm[c * n + _brev(i, logn)] = work[base + i * n + c] * f
        _df_stages(sm, kb, n, logn, tw, conj)
        sh = 0 if sref == ZERO_ROW else sref
        for e in range(n * kb):
            i, c = e // kb, e % kb
            S[base + i * n + c] = sm[c * n + i] * 2.0 ** sh
    return S.reshape(n, n, n), written.reshape(n, n, n)


def _df_c2r(B, S, sign):
    """fft_cols_f64_kernel on the columns m' < B, then fft_rows_c2r_kernel."""
    n, N, _, rpb, kb = _df_shapes(B)
    logn, logN, conj = n.bit_length() - 1, N.bit_length() - 1, sign < 0
    tw = np.exp(2j * np.pi * np.arange(n // 2) / n)
    twN = tw[0:2 * (N >> 1):2]
    Sf = S.reshape(-1)
    work = np.full(n ** 3, np.nan + 0j)
    cexp = np.full(n * N, 7777)
    tiles = N // kb
    for blk in range(n * tiles):
        js, k0 = blk // tiles, (blk % tiles) * kb
        base = js * n * n + k0
        sm = np.full(kb * n, np.nan + 0j)
        cmax = [0] * kb
        for e in range(n * kb):
            i, c = e // kb, e % kb
            v = Sf[base + i * n + c]
            cmax[c] = max(cmax[c], _exp_of(v))
            sm[c * n + _brev(i, logn)] = v
        for e in range(n * kb):
            i, c = e // kb, e % kb
            sm[c * n + _brev(i, logn)] *= 2.0 ** ((1023 - cmax[c]) if cmax[c] else 0)
        for t in range(kb):
            assert js * N + k0 + t < n * N
            cexp[js * N + k0 + t] = cmax[t] - 1023 if cmax[t] else ZERO_ROW
        _df_stages(sm, kb, n, logn, tw, conj)
        for e in range(n * kb):
            i, c = e // kb, e % kb
            work[base + i * n + c] = sm[c * n + i]
    out = np.full(n ** 3, np.nan)
    nrows = n * n
    assert n % rpb == 0
    for blk in range(nrows // rpb):
        r0 = blk * rpb
        js, rows = r0 // n, min(rpb, nrows - r0)
        assert (r0 + rows - 1) // n == js  # a block's rows lie in one slice
        sref = max(cexp[js * N + k] for k in range(N))
        fs = [0.0 if cexp[js * N + k] - sref < -126 else 2.0 ** (cexp[js * N + k] - sref) for k in range(N)]
        sm = np.full(rpb * N, np.nan + 0j)
        for e in range(rows * N):
            rl, k = e >> logN, e & (N - 1)
            row = (r0 + rl) * n
            a = work[row + k] * fs[k]
            b = work[row + N - k] * fs[N - k] if k else 0j
            A = complex(a.real + b.real, a.imag - b.imag)
            D = complex(a.real - b.real, a.imag + b.imag)
            C = (np.conj(tw[k]) if conj else tw[k]) * D
            sm[rl * N + _brev(k, logN)] = A + 1j * C
        _df_stages(sm, rows, N, logN, twN, conj)
        sh = 0 if sref == ZERO_ROW else sref
        for e in range(rows * N):
            o = r0 * N + e
            assert 2 * o + 1 < n ** 3
            out[2 * o], out[2 * o + 1] = sm[e].real * 2.0 ** sh, sm[e].imag * 2.0 ** sh
    return out.reshape(n, n, n)


@pytest.mark.parametrize("B", [2, 4, 8, 16])
def test_df_real_forward_model_matches_numpy(B):
    n = 2 * B
    rng = np.random.default_rng(900 + B)
    x = rng.standard_normal((n, n, n)) * np.exp(rng.uniform(-30, 30, size=(n, n, 1)))  # rows of mixed scales
    x[1] = 0.0          # an all-zero slice: the zero-row branch
    S, written = _df_r2c(B, x, +1)
    ref = np.fft.ifft2(x, axes=(1, 2)) * n * n  # exp(+i ...), unnormalised
    assert np.isnan(S[:, :, B:]).all()          # the columns m' >= B are never written
    assert (written[:, :, :B] == 1).all() and (written[:, :, B:] == 0).all()
    err = np.linalg.norm(S[:, :, :B] - ref[:, :, :B]) / np.linalg.norm(ref[:, :, :B])
    assert err < 1e-13


@pytest.mark.parametrize("B", [2, 4, 8, 16])
def test_df_real_inverse_model_matches_numpy(B):
    n = 2 * B
    rng = np.random.default_rng(950 + B)
    X = np.fft.fft2(rng.standard_normal((n, n, n)), axes=(1, 2))
    X[:, :, B] = 0.0    # the m' = -B column and m = -B row, cleared as the iDWT leaves them
    X[:, B, :] = 0.0
    X *= np.exp(rng.uniform(-30, 30, size=(n, 1, 1)))
    X[2] = 0.0          # an all-zero slice
    want = np.fft.fft2(X, axes=(1, 2))  # exp(-i ...): real up to rounding
    assert np.abs(want.imag).max() <= 1e-12 * np.abs(want).max()
    S = X.copy()
    S[:, :, B:] = np.nan  # the kernels must not read the columns m' >= B
    g = _df_c2r(B, S, -1)
    assert np.isfinite(g).all()
    assert np.linalg.norm(g - want.real) <= 1e-13 * np.linalg.norm(want.real)


def test_df_real_launch_shapes():
    """For every power-of-two B the host code accepts (2..512): the r2c row
    blocks stay within the 256-entry row-maximum array, the c2r row blocks
    divide a slice, the column tiles divide B and fit the 64-entry column
    array, shared memory fits, and every grid is below 2^31 blocks."""
    for lb in range(1, 10):
        B = 1 << lb
        n, N, rpb_r, rpb_c, kb = _df_shapes(B)
        assert 1 <= rpb_r <= 256 and 1 <= rpb_c and n % rpb_c == 0
        assert N % kb == 0 and kb <= 64
        rbytes = 16 * (N + N // 2 + max(rpb_r, rpb_c) * N)
        cbytes = 16 * (n // 2 + kb * n)
        assert rbytes <= 227 * 1024 and cbytes <= 227 * 1024
        assert (n * n + rpb_r - 1) // rpb_r < 2 ** 31 and n * (N // kb) < 2 ** 31
        assert rpb_r * N <= 4096 and rpb_c * N <= 4096
