"""FP64 CPU oracle for the SO(3) Fourier transform (test infrastructure only).

This package is the plain, slow, obviously-correct reference that the CUDA
library is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library itself never does.
It shares no code with the CUDA path.  The arithmetic lives in
``soft_oracle.c`` (plain C, compiled here with gcc); this module only marshals
numpy arrays.

Every function follows Sec. 2 of Lux, Wuelker, Chirikjian, "Parallelization of
the FFT on SO(3)" (arXiv:1808.00896):

* ``weights``                 -- Eq. (weights)
* ``wigner_d_explicit``       -- the explicit Jacobi form (Sec. 2.2), extended
                                 to all (m, m') by the beta-preserving symmetries
                                 of Eq. (Wigner_symmetries)
* ``wigner_d_column``         -- Eq. (Wigner_d_recurrence) from the four seeds
* ``forward`` / ``inverse``   -- the sequential fast transform of Sec. 2.4:
                                 2-D DFT per beta slice, then the DWT
                                 V_B T_B W_B per (m, m'); inverse T_B^T then DFT
* ``direct_forward`` / ``direct_inverse`` -- Eq. (quadrature) and
                                 Eq. (fourier_representation) summed directly,
                                 O(B^6), small B only
* ``forward_pairs`` / ``inverse_points`` -- sampled forms for large B
* ``correlation_coeffs`` / ``correlation`` / ``argmax_real`` -- rotational
                                 correlation of two spherical functions (the
                                 rotational matching application of Sec. 1):
                                 c(l,m,m') = g_lm conj(f_lm'), then ``inverse``
* ``forward_adjoint`` / ``inverse_adjoint`` -- the adjoints of the two
                                 transforms: E^H W T^T V and T E (E the
                                 per-slice DFT with exp(+i))
* ``set_threads``             -- OpenMP threads for the loops over independent
                                 order pairs, slices, sampled pairs and points
                                 (1 by default; results do not depend on it)
* ``forward_strided`` / ``inverse_strided`` -- timing samples: every
                                 stride-th beta slice and row m of order pairs
                                 only (not a transform; used to time the oracle
                                 at sizes where a full run takes too long)

Every function is pinned by tests in ``tests/test_oracle_*.py`` to closed
forms, a textbook routine (sympy's Wigner-d, scipy's Jacobi polynomials),
orthogonality, exact quadrature, Parseval, one-hot and round-trip identities.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "soft_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile soft_oracle.c into liboracle.so with gcc (no fast-math), with
    OpenMP when the compiler has it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        c_int, c_double, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "oracle_beta": (c_double, [c_int, c_int]),
            "oracle_alpha": (c_double, [c_int, c_int]),
            "oracle_weights": (None, [c_int, dp]),
            "oracle_jacobi": (c_double, [c_int, c_int, c_int, c_double]),
            "oracle_wigner_d_explicit": (c_double, [c_int, c_int, c_int, c_double]),
            "oracle_wigner_seed": (c_double, [c_int, c_int, c_double]),
            "oracle_wigner_d_column": (None, [c_int, c_int, c_int, c_double, dp]),
            "oracle_num_coeffs": (c_i64, [c_int]),
            "oracle_coef_index": (c_i64, [c_int, c_int, c_int, c_int]),
            "oracle_dft1": (None, [c_int, dp, c_int, c_int]),
            "oracle_dft2_slices": (None, [c_int, c_int, dp, c_int]),
            "oracle_forward": (c_int, [c_int, dp, dp]),
            "oracle_inverse": (c_int, [c_int, dp, dp]),
            "oracle_forward_strided": (c_int, [c_int, dp, dp, c_int]),
            "oracle_inverse_strided": (c_int, [c_int, dp, dp, c_int]),
            "oracle_set_threads": (None, [c_int]),
            "oracle_get_threads": (c_int, []),
            "oracle_openmp": (c_int, []),
            "oracle_direct_forward": (c_int, [c_int, dp, dp]),
            "oracle_direct_inverse": (c_int, [c_int, dp, dp]),
            "oracle_forward_pairs": (c_int, [c_int, dp, c_int, ip, dp]),
            "oracle_forward_adjoint": (c_int, [c_int, dp, dp]),
            "oracle_correlation_coeffs": (c_int, [c_int, dp, dp, dp]),
            "oracle_inverse_adjoint": (c_int, [c_int, dp, dp]),
            "oracle_inverse_points": (c_int, [c_int, dp, c_int, ip, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def set_threads(n: int) -> int:
    """Threads for the oracle's parallel loops (over order pairs, beta slices,
    sampled pairs and sampled points); returns the previous count.  Without
    OpenMP the loops stay serial whatever is set."""
    lib = _load()
    prev = int(lib.oracle_get_threads())
    lib.oracle_set_threads(int(n))
    return prev


def threads() -> int:
    """Threads the parallel loops use (1 when built without OpenMP)."""
    lib = _load()
    return int(lib.oracle_get_threads()) if lib.oracle_openmp() else 1


def openmp() -> bool:
    return bool(_load().oracle_openmp())


def num_coeffs(B: int) -> int:
    """B(4B^2-1)/3 coefficients f(l,m,m') with l < B (Sec. 2.4)."""
    return int(_load().oracle_num_coeffs(B))


def coef_index(B: int, l: int, m: int, mp: int) -> int:
    """Offset of f(l,m,m') in the coefficient array; -1 if out of range."""
    return int(_load().oracle_coef_index(B, l, m, mp))


def beta(B: int) -> np.ndarray:
    """beta_j = (2j+1) pi / (4B), j < 2B (Eq. quadrature)."""
    return np.array([_load().oracle_beta(B, j) for j in range(2 * B)])


def weights(B: int) -> np.ndarray:
    """Quadrature weights w_B(j), j < 2B (Eq. weights)."""
    w = np.zeros(2 * B)
    _load().oracle_weights(B, _dp(w))
    return w


def jacobi(n: int, a: int, b: int, x: float) -> float:
    return float(_load().oracle_jacobi(n, a, b, x))


def wigner_d_explicit(l: int, m: int, mp: int, beta_: float) -> float:
    """d(l,m,m';beta) from the explicit Jacobi form (Sec. 2.2)."""
    return float(_load().oracle_wigner_d_explicit(l, m, mp, beta_))


def wigner_seed(m: int, mp: int, beta_: float) -> float:
    """d(l0,m,m';beta), l0 = max(|m|,|m'|), from the paper's initial cases."""
    return float(_load().oracle_wigner_seed(m, mp, beta_))


def wigner_d_column(B: int, m: int, mp: int, beta_: float) -> np.ndarray:
    """[d(l,m,m';beta)] for l = max(|m|,|m'|)..B-1 by Eq. (Wigner_d_recurrence)."""
    l0 = max(abs(m), abs(mp))
    out = np.zeros(max(B - l0, 0))
    if B - l0 > 0:
        _load().oracle_wigner_d_column(B, m, mp, beta_, _dp(out))
    return out


def dft2_slices(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 2-D DFT with exp(sign*2*pi*i*...) on each trailing n x n slice."""
    x = _as_c128(x).copy()
    n = x.shape[-1]
    ns = x.size // (n * n)
    _load().oracle_dft2_slices(ns, n, _dp(x.view(np.float64)), sign)
    return x


def dft1(x: np.ndarray, sign: int) -> np.ndarray:
    x = _as_c128(x).copy()
    _load().oracle_dft1(x.size, _dp(x.view(np.float64)), 1, sign)
    return x


def _check_grid(B: int, grid) -> np.ndarray:
    g = _as_c128(grid)
    n = 2 * B
    if g.size != n ** 3:
        raise ValueError(f"grid must hold (2B)^3 = {n ** 3} complex values, got {g.size}")
    return g


def _check_coef(B: int, coef) -> np.ndarray:
    c = _as_c128(coef)
    if c.size != num_coeffs(B):
        raise ValueError(f"coef must hold B(4B^2-1)/3 = {num_coeffs(B)} values, got {c.size}")
    return c


def forward(B: int, grid) -> np.ndarray:
    """Sequential fast forward transform (Sec. 2.4): grid[j][i][k] -> coefficients."""
    g = _check_grid(B, grid)
    out = np.zeros(num_coeffs(B), dtype=np.complex128)
    rc = _load().oracle_forward(B, _dp(g.view(np.float64)), _dp(out.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_forward failed ({rc})")
    return out


def inverse(B: int, coef) -> np.ndarray:
    """Sequential fast inverse transform (Sec. 2.4): coefficients -> grid[j][i][k]."""
    c = _check_coef(B, coef)
    n = 2 * B
    out = np.zeros((n, n, n), dtype=np.complex128)
    rc = _load().oracle_inverse(B, _dp(c.view(np.float64)), _dp(out.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_inverse failed ({rc})")
    return out


def forward_strided(B: int, grid, stride: int, out: np.ndarray | None = None) -> np.ndarray:
    """TIMING SAMPLE of ``forward``: only the beta slices j with j % stride
    == 0 and the rows m of order pairs with (m + B - 1) % stride == stride // 2
    are processed: about 1/stride of the per-slice and per-pair work, plus the
    full run's fixed costs (the copy of the grid).  A stride above 4B leaves
    the fixed costs alone.  Not a transform."""
    g = _check_grid(B, grid)
    if out is None:
        out = np.zeros(num_coeffs(B), dtype=np.complex128)
    rc = _load().oracle_forward_strided(B, _dp(g.view(np.float64)), _dp(out.view(np.float64)), int(stride))
    if rc:
        raise RuntimeError(f"oracle_forward_strided failed ({rc})")
    return out


def inverse_strided(B: int, coef, stride: int, out: np.ndarray | None = None) -> np.ndarray:
    """TIMING SAMPLE of ``inverse`` (see ``forward_strided``)."""
    c = _check_coef(B, coef)
    n = 2 * B
    if out is None:
        out = np.zeros((n, n, n), dtype=np.complex128)
    rc = _load().oracle_inverse_strided(B, _dp(c.view(np.float64)), _dp(out.view(np.float64)), int(stride))
    if rc:
        raise RuntimeError(f"oracle_inverse_strided failed ({rc})")
    return out


def direct_forward(B: int, grid) -> np.ndarray:
    """Eq. (quadrature) summed term by term, O(B^6)."""
    if B > 10:
        raise ValueError("direct_forward is O(B^6); use B <= 10")
    g = _check_grid(B, grid)
    out = np.zeros(num_coeffs(B), dtype=np.complex128)
    _load().oracle_direct_forward(B, _dp(g.view(np.float64)), _dp(out.view(np.float64)))
    return out


def direct_inverse(B: int, coef) -> np.ndarray:
    """Eq. (fourier_representation) summed term by term at every grid point, O(B^6)."""
    if B > 10:
        raise ValueError("direct_inverse is O(B^6); use B <= 10")
    c = _check_coef(B, coef)
    n = 2 * B
    out = np.zeros((n, n, n), dtype=np.complex128)
    _load().oracle_direct_inverse(B, _dp(c.view(np.float64)), _dp(out.view(np.float64)))
    return out


def forward_adjoint(B: int, coef) -> np.ndarray:
    """Adjoint of ``forward``: coefficients -> grid, E^H W T^T V."""
    c = _check_coef(B, coef)
    n = 2 * B
    out = np.zeros((n, n, n), dtype=np.complex128)
    rc = _load().oracle_forward_adjoint(B, _dp(c.view(np.float64)), _dp(out.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_forward_adjoint failed ({rc})")
    return out


def inverse_adjoint(B: int, grid) -> np.ndarray:
    """Adjoint of ``inverse``: grid -> coefficients, T E."""
    g = _check_grid(B, grid)
    out = np.zeros(num_coeffs(B), dtype=np.complex128)
    rc = _load().oracle_inverse_adjoint(B, _dp(g.view(np.float64)), _dp(out.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_inverse_adjoint failed ({rc})")
    return out


def correlation_coeffs(B: int, f_sh, g_sh) -> np.ndarray:
    """c(l,m,m') = g_lm conj(f_lm') for spherical-harmonic vectors of length B^2
    (index l*l + m + l); the inverse transform of c is C(R) = <g(R^-1 .), f>."""
    f = _as_c128(f_sh)
    g = _as_c128(g_sh)
    if f.size != B * B or g.size != B * B:
        raise ValueError("spherical-harmonic vectors must hold B^2 values")
    out = np.zeros(num_coeffs(B), dtype=np.complex128)
    _load().oracle_correlation_coeffs(B, _dp(f.view(np.float64)), _dp(g.view(np.float64)),
                                      _dp(out.view(np.float64)))
    return out


def correlation(B: int, f_sh, g_sh) -> np.ndarray:
    """C(alpha_i, beta_j, gamma_k) on the (2B)^3 grid, layout [j][i][k]."""
    return inverse(B, correlation_coeffs(B, f_sh, g_sh))


def argmax_real(values) -> tuple[int, float]:
    """Linear index and value of the largest real part (first index on ties)."""
    v = np.asarray(values).reshape(-1).real
    i = int(np.argmax(v))
    return i, float(v[i])


def forward_pairs(B: int, grid, pairs) -> list[np.ndarray]:
    """Forward coefficients of the given (m, m') pairs only; one array per pair
    holding l = max(|m|,|m'|)..B-1."""
    g = _check_grid(B, grid)
    pairs = [(int(m), int(mp)) for m, mp in pairs]
    if any(max(abs(m), abs(mp)) >= B for m, mp in pairs):
        raise ValueError("every order pair needs |m|, |m'| < B")
    flat = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
    lens = [B - max(abs(m), abs(mp)) for m, mp in pairs]
    out = np.zeros(sum(lens), dtype=np.complex128)
    rc = _load().oracle_forward_pairs(B, _dp(g.view(np.float64)), len(pairs), _ip(flat),
                                      _dp(out.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_forward_pairs failed ({rc})")
    res, o = [], 0
    for L in lens:
        res.append(out[o:o + L].copy())
        o += L
    return res


def inverse_points(B: int, coef, points) -> np.ndarray:
    """Inverse transform evaluated at grid points (i, j, k) only."""
    c = _check_coef(B, coef)
    flat = np.ascontiguousarray(np.array(points, dtype=np.int32).reshape(-1))
    if flat.size % 3 or (flat.size and (flat.min() < 0 or flat.max() >= 2 * B)):
        raise ValueError("grid points are (i, j, k) triples with 0 <= i, j, k < 2B")
    out = np.zeros(len(flat) // 3, dtype=np.complex128)
    rc = _load().oracle_inverse_points(B, _dp(c.view(np.float64)), len(out), _ip(flat),
                                       _dp(out.view(np.float64)))
    if rc:
        raise RuntimeError(f"oracle_inverse_points failed ({rc})")
    return out


def coef_lmm(B: int) -> np.ndarray:
    """(l, m, m') of every entry of the coefficient array, by plain counting."""
    rows = []
    for m in range(1 - B, B):
        for mp in range(1 - B, B):
            for l in range(max(abs(m), abs(mp)), B):
                rows.append((l, m, mp))
    return np.array(rows, dtype=np.int64).reshape(-1, 3)
