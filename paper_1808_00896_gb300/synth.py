"""Seeded synthetic inputs for the SO(3) transforms.

This module holds random-number plumbing and index bookkeeping only; none of
the transform's arithmetic.  Both the CUDA path's tests/benchmark and the CPU
oracle draw their inputs from here, so that the two sides see identical bytes.

Recipes (the paper's own benchmark inputs are not described in the available
text, so these are synthetic stand-ins with the sizes of its workloads):

* ``"uniform"``     -- real and imaginary parts iid U(-1, 1)
* ``"gauss_decay"`` -- iid complex Gaussian (re, im ~ N(0, 1)) scaled by 1/(l+1),
                       a smooth band-limited function
* ``random_grid``   -- iid U(-1, 1) samples on the (2B)^3 Euler grid (not
                       band-limited; the forward transform is still the
                       quadrature sum of Eq. (quadrature) applied to it)

Coefficient layout: for m = 1-B..B-1 (outer), m' = 1-B..B-1 (inner), the run
l = max(|m|,|m'|)..B-1 is contiguous.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 0x5F3F1808


def num_coeffs(B: int) -> int:
    return B * (4 * B * B - 1) // 3


def coef_degrees(B: int) -> np.ndarray:
    """Degree l of every entry of the coefficient array (int32)."""
    r = np.arange(1 - B, B)
    l0 = np.maximum(np.abs(r)[:, None], np.abs(r)[None, :]).reshape(-1)
    lens = (B - l0).astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    total = int(lens.sum())
    idx = np.arange(total, dtype=np.int64)
    l = np.repeat(l0.astype(np.int64), lens) + (idx - np.repeat(starts, lens))
    return l.astype(np.int32)


def coefficients(B: int, kind: str = "gauss_decay", seed: int = BASE_SEED) -> np.ndarray:
    """Random coefficient vector (complex128, length B(4B^2-1)/3)."""
    rng = np.random.default_rng(seed)
    n = num_coeffs(B)
    if kind == "uniform":
        c = np.empty(n, dtype=np.complex128)
        v = c.view(np.float64)
        v[:] = rng.uniform(-1.0, 1.0, size=2 * n)
        return c
    if kind == "gauss_decay":
        c = np.empty(n, dtype=np.complex128)
        v = c.view(np.float64)
        v[:] = rng.standard_normal(size=2 * n)
        c *= 1.0 / (coef_degrees(B).astype(np.float64) + 1.0)
        return c
    raise ValueError(f"unknown coefficient kind {kind!r}")


def sh_coefficients(B: int, seed: int = BASE_SEED) -> np.ndarray:
    """Spherical-harmonic coefficients of a random band-limited function on the
    sphere: f_lm (index l*l + m + l, l < B), iid complex Gaussian x 1/(l+1)."""
    rng = np.random.default_rng(seed)
    c = np.empty(B * B, dtype=np.complex128)
    c.view(np.float64)[:] = rng.standard_normal(2 * B * B)
    l = np.floor(np.sqrt(np.arange(B * B))).astype(np.float64)
    return c / (l + 1.0)


def correlation_requests(count: int = 64, bandwidths=(8, 16, 32, 64, 128), seed: int = BASE_SEED):
    """Batched rotational-matching workload: `count` requests with bandwidths
    drawn uniformly from `bandwidths`, each a pair (f_lm, g_lm) of random
    band-limited spherical functions.  Returns a list of (B, f_sh, g_sh)."""
    rng = np.random.default_rng(seed)
    Bs = rng.choice(np.asarray(bandwidths), size=count)
    return [(int(B), sh_coefficients(int(B), seed + 2 * i + 1), sh_coefficients(int(B), seed + 2 * i + 2))
            for i, B in enumerate(Bs)]


def random_grid(B: int, seed: int = BASE_SEED) -> np.ndarray:
    """iid U(-1,1) complex samples on the (2B)^3 grid, shape (2B, 2B, 2B) = [j][i][k]."""
    rng = np.random.default_rng(seed)
    n = 2 * B
    g = np.empty((n, n, n), dtype=np.complex128)
    g.view(np.float64)[...] = rng.uniform(-1.0, 1.0, size=(n, n, 2 * n))
    return g


def rel_l2(x, ref) -> float:
    """||x - ref||_2 / ||ref||_2 over all complex entries."""
    x = np.asarray(x).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))
