"""Real grids: soft_forward_real / soft_inverse_real against the oracle.

A real function on SO(3) has f(l,-m,-m') = (-1)^(m-m') conj f(l,m,m') (the
symmetries of Eq. (Wigner_symmetries)); the real entry points contract one
partner of each such conjugate pair.  The oracle has no real mode: it runs the
complex transforms on the same data (zero imaginary parts in, real part out),
so every comparison here is against the plain definition.  Bound: rel-L2
<= 1e-10, as the FP64 path, for FP64 and FP64-TC plans alike (FP64 plans run
the half-spectrum slice FFT in FP64, FP64-TC plans from B = 2 on in
double-float arithmetic, and their kernels contract the even partners on the
tensor cores).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, capi, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def real_grid(B, seed):
    return np.ascontiguousarray(synth.random_grid(B, seed=seed).real)


def runs(B):
    """(m, m', start, length) of every coefficient run."""
    out = []
    for m in range(1 - B, B):
        for mp in range(1 - B, B):
            l0 = max(abs(m), abs(mp))
            out.append((m, mp, oracle.coef_index(B, l0, m, mp), B - l0))
    return out


def symmetrize(B, c):
    """The coefficients of a real function: f(l,-m,-m') = (-1)^(m-m') conj f(l,m,m')."""
    c = c.copy()
    for m, mp, o, L in runs(B):
        if (m, mp) == (0, 0):
            c[o:o + L] = c[o:o + L].real
        elif (m, mp) > (-m, -mp):
            o2 = oracle.coef_index(B, max(abs(m), abs(mp)), -m, -mp)
            c[o:o + L] = (-1.0) ** (m - mp) * np.conj(c[o2:o2 + L])
    return c


def odd_partner(m, mp):
    """True when (m, m') is the second of its conjugate pair in the cluster's
    partner order: (m,m'),(-m,-m') | (m',m),(-m',-m) | (-m,m'),(m,-m') |
    (-m',m),(m',-m) for a representative m >= m' >= 0."""
    a, b = max(abs(m), abs(mp)), min(abs(m), abs(mp))
    if a == 0:
        return False
    if b == 0:
        order = [(a, 0), (-a, 0), (0, a), (0, -a)]
    elif a == b:
        order = [(a, a), (-a, -a), (-a, a), (a, -a)]
    else:
        order = [(a, b), (-a, -b), (b, a), (-b, -a), (-a, b), (a, -b), (-b, a), (b, -a)]
    return order.index((m, mp)) % 2 == 1


POW2_B = [1, 2, 4, 8, 16, 32, 64, 128]
MODES = ["fp64", "fp64_tc"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("B", POW2_B)
def test_forward_real_parity(B, mode):
    g = real_grid(B, 8100 + B)
    want = oracle.forward(B, g.astype(np.complex128))
    with Plan(B, mode, device=DEV) as p:
        f = p.forward_real(torch.from_numpy(g).to(DEV)).cpu().numpy()
        p.sync()
    assert np.isfinite(f).all()
    assert synth.rel_l2(f, want) < TOL


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("B", POW2_B)
def test_inverse_real_parity(B, mode):
    c = symmetrize(B, synth.coefficients(B, "gauss_decay", seed=8200 + B))
    want = oracle.inverse(B, c)
    assert np.linalg.norm(want.imag) <= 1e-12 * np.linalg.norm(want.real)  # the oracle agrees it is real
    with Plan(B, mode, device=DEV) as p:
        g = p.inverse_real(torch.from_numpy(c).to(DEV)).cpu().numpy()
        p.sync()
    assert g.dtype == np.float64 and np.isfinite(g).all()
    assert synth.rel_l2(g, want.real) < TOL


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("B", [4, 16])
def test_forward_real_output_is_exactly_symmetric(B, mode):
    g = real_grid(B, 8300 + B)
    with Plan(B, mode, device=DEV) as p:
        f = p.forward_real(torch.from_numpy(g).to(DEV)).cpu().numpy()
        p.sync()
    for m, mp, o, L in runs(B):
        o2 = oracle.coef_index(B, max(abs(m), abs(mp)), -m, -mp)
        if (m, mp) != (0, 0):
            assert np.array_equal(f[o:o + L], (-1.0) ** (m - mp) * np.conj(f[o2:o2 + L])), (m, mp)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("B", [2, 8, 32])
def test_inverse_real_reads_one_partner_per_pair(B, mode):
    """The second partner of every conjugate pair is never read: NaN there
    leaves the result unchanged."""
    c = symmetrize(B, synth.coefficients(B, "uniform", seed=8400 + B))
    poisoned = c.copy()
    count = 0
    for m, mp, o, L in runs(B):
        if odd_partner(m, mp):
            poisoned[o:o + L] = complex(np.nan, np.nan)
            count += L
    assert count == (len(c) - B) // 2  # all but the self-conjugate (0, 0) run, halved
    with Plan(B, mode, device=DEV) as p:
        g = p.inverse_real(torch.from_numpy(c).to(DEV)).cpu().numpy()
        h = p.inverse_real(torch.from_numpy(poisoned).to(DEV)).cpu().numpy()
        p.sync()
    assert np.array_equal(g, h)


@pytest.mark.parametrize("mode", MODES)
def test_round_trip_band_limited_real(mode):
    B = 32
    c = symmetrize(B, synth.coefficients(B, "gauss_decay", seed=8500))
    g = np.ascontiguousarray(oracle.inverse(B, c).real)
    with Plan(B, mode, device=DEV) as p:
        f = p.forward_real(torch.from_numpy(g).to(DEV)).cpu().numpy()
        back = p.inverse_real(torch.from_numpy(f).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, c) < TOL
    assert synth.rel_l2(back, g) < TOL


@pytest.mark.parametrize("mode", MODES)
def test_sampled_real_B256(mode):
    """Full size: sampled order pairs of the forward (both partners of a
    conjugate pair) against the oracle's one-by-one form."""
    B = 256
    rng = np.random.default_rng(8600)
    g = real_grid(B, 8601)
    with Plan(B, mode, device=DEV) as p:
        f = p.forward_real(torch.from_numpy(g).to(DEV)).cpu().numpy()
        p.sync()
    pairs = []
    for _ in range(5):
        m, mp = (int(v) for v in rng.integers(1 - B, B, size=2))
        pairs += [(m, mp), (-m, -mp)]
    want = oracle.forward_pairs(B, g.astype(np.complex128), pairs)
    got = [f[oracle.coef_index(B, max(abs(m), abs(mp)), m, mp):][:B - max(abs(m), abs(mp))] for m, mp in pairs]
    assert synth.rel_l2(np.concatenate(got), np.concatenate(want)) < TOL


@pytest.mark.parametrize("B,mode", [(3, "fp64"), (3, "fp64_tc"), (8, "bf16x3")])
def test_real_entry_points_unsupported(B, mode):
    """Real entry points need an FP64 or FP64-TC plan with power-of-two 2B."""
    with Plan(B, mode, device=DEV) as p:
        g = torch.zeros((2 * B,) * 3, dtype=torch.float64, device=DEV)
        c = p.empty_coef()
        assert capi.soft_forward_real(p.handle, g.data_ptr(), c.data_ptr(), 0) == capi.SOFT_ERR_UNSUPPORTED
        assert capi.soft_inverse_real(p.handle, c.data_ptr(), g.data_ptr(), 0) == capi.SOFT_ERR_UNSUPPORTED


@pytest.mark.parametrize("scale", [1e-150, 1e150])
def test_fp64tc_real_inputs_far_outside_the_fp32_range(scale):
    """The double-float half-spectrum FFT scales every row (forward) or
    column (inverse) by the power of two of its largest magnitude, so grids
    and coefficients far outside the FP32 exponent range keep the bound."""
    B = 16
    g = real_grid(B, 8700) * scale
    c = symmetrize(B, synth.coefficients(B, "gauss_decay", seed=8701)) * scale
    with Plan(B, "fp64_tc", device=DEV) as p:
        f = p.forward_real(torch.from_numpy(g).to(DEV)).cpu().numpy()
        back = p.inverse_real(torch.from_numpy(c).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, g.astype(np.complex128))) < TOL
    assert synth.rel_l2(back, oracle.inverse(B, c).real) < TOL


def test_fp64tc_real_zero_slices_and_rows():
    """All-zero rows and slices take the zero-scale branch of the row and
    column scales; the rest of the grid must be unaffected."""
    B = 8
    g = real_grid(B, 8800)
    g[3] = 0.0           # one whole beta slice
    g[5, 2] = 0.0        # one row of another slice
    c = symmetrize(B, synth.coefficients(B, "gauss_decay", seed=8801))
    with Plan(B, "fp64_tc", device=DEV) as p:
        f = p.forward_real(torch.from_numpy(g).to(DEV)).cpu().numpy()
        z = p.forward_real(torch.zeros((2 * B,) * 3, dtype=torch.float64, device=DEV)).cpu().numpy()
        back = p.inverse_real(torch.from_numpy(c).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(f, oracle.forward(B, g.astype(np.complex128))) < TOL
    assert np.all(z == 0)
    assert synth.rel_l2(back, oracle.inverse(B, c).real) < TOL


def test_fp64tc_real_B512_against_the_fp64_path():
    """Every coefficient and grid value of the real-grid calls at B = 512
    (1024^3 grid; the double-float FFT's largest row and column shapes)
    against the FP64 plan's real-grid calls, whose agreement with the oracle
    the smaller and sampled cases establish.  Norms on the device."""
    B = 512
    gen = torch.Generator(device=DEV).manual_seed(8900)
    g = torch.randn((2 * B,) * 3, dtype=torch.float64, device=DEV, generator=gen)
    # the real-grid inverse reads one partner of each conjugate pair, the same in both plans
    c = torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=8901)).to(DEV)

    def rel(x, ref):
        return (torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)).item()

    with Plan(B, "fp64", device=DEV) as a:
        fa = a.forward_real(g)
        ga = a.inverse_real(c)
        a.sync()
    with Plan(B, "fp64_tc", device=DEV) as b:
        fb = b.forward_real(g)
        gb = b.inverse_real(c)
        b.sync()
    del g
    assert rel(fb, fa) < TOL
    assert rel(gb, ga) < TOL
