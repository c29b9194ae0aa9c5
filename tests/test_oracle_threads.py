"""The oracle's OpenMP loops: every order pair, slice, sampled pair or point
is computed by one thread in the written order, so the results are
bit-identical for any thread count; the strided timing samples touch only
the order pairs of the sampled rows m."""
import numpy as np
import pytest

import oracle
from paper_1808_00896_gb300 import synth


@pytest.fixture
def threads4():
    prev = oracle.set_threads(4)
    yield
    oracle.set_threads(prev)


@pytest.mark.parametrize("B", [6, 8])
def test_results_do_not_depend_on_threads(B):
    grid = synth.random_grid(B, seed=900 + B)
    coef = synth.coefficients(B, "uniform", seed=910 + B)
    pairs = [(0, 0), (B - 1, 1 - B), (2, -3), (-1, 1)]
    pts = [(0, 0, 0), (1, 2, 3), (2 * B - 1, B, 0)]
    prev = oracle.set_threads(1)
    try:
        ref = (oracle.forward(B, grid), oracle.inverse(B, coef), oracle.forward_pairs(B, grid, pairs),
               oracle.inverse_points(B, coef, pts))
        oracle.set_threads(4)
        got = (oracle.forward(B, grid), oracle.inverse(B, coef), oracle.forward_pairs(B, grid, pairs),
               oracle.inverse_points(B, coef, pts))
    finally:
        oracle.set_threads(prev)
    assert np.array_equal(ref[0], got[0])
    assert np.array_equal(ref[1], got[1])
    for a, b in zip(ref[2], got[2]):
        assert np.array_equal(a, b)
    assert np.array_equal(ref[3], got[3])


def test_stride_one_is_the_transform(threads4):
    B = 7
    grid = synth.random_grid(B, seed=920)
    coef = synth.coefficients(B, "uniform", seed=921)
    assert np.array_equal(oracle.forward_strided(B, grid, 1), oracle.forward(B, grid))
    assert np.array_equal(oracle.inverse_strided(B, coef, 1), oracle.inverse(B, coef))


def test_strided_sample_touches_only_sampled_pairs(threads4):
    B, stride = 8, 5
    grid = synth.random_grid(B, seed=930)
    out = oracle.forward_strided(B, grid, stride)
    R = 2 * B - 1
    for p in range(R * R):
        m, mp = p // R + 1 - B, p % R + 1 - B
        l0 = max(abs(m), abs(mp))
        run = out[oracle.coef_index(B, l0, m, mp):oracle.coef_index(B, l0, m, mp) + B - l0]
        if (m + B - 1) % stride != stride // 2:
            assert not run.any(), (m, mp)
        else:
            assert np.all(run != 0), (m, mp)


def test_sampled_forms_reject_out_of_range_indices():
    B = 4
    grid = synth.random_grid(B, seed=940)
    coef = synth.coefficients(B, "uniform", seed=941)
    with pytest.raises(ValueError):
        oracle.forward_pairs(B, grid, [(0, 0), (B, 0)])
    with pytest.raises(ValueError):
        oracle.inverse_points(B, coef, [(0, 0, 2 * B)])
