"""The Clenshaw iDWT (the last iDWT variant of FP64 plans): the sum over the
degrees runs backwards by Clenshaw's algorithm instead of generating each
Wigner-d value by the forward recurrence.  Against the oracle's inverse, its
adjoint-of-forward (V and W applied) and on real grids, at B = 1..128 in full
and B = 256 on sampled grid points."""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _clenshaw(p):
    p.set_variant(1, p.num_variants(1) - 1)
    return p


@pytest.mark.parametrize("B", [1, 2, 3, 8, 16, 17, 33, 64, 128])
def test_clenshaw_inverse_and_adjoint_match_oracle(B):
    coef = synth.coefficients(B, "gauss_decay", seed=8800 + B)
    with _clenshaw(Plan(B, device=DEV)) as p:
        c = torch.from_numpy(coef).to(DEV)
        g = p.inverse(c).cpu().numpy()
        a = p.forward_adjoint(c).cpu().numpy()
        p.sync()
    assert np.isfinite(g).all() and np.isfinite(a).all()
    assert synth.rel_l2(g, oracle.inverse(B, coef)) < TOL
    assert synth.rel_l2(a, oracle.forward_adjoint(B, coef)) < TOL


@pytest.mark.parametrize("B", [4, 32, 64])
def test_clenshaw_real_grid(B):
    coef = synth.coefficients(B, "gauss_decay", seed=8900 + B)
    c_sym = oracle.forward(B, oracle.inverse(B, coef).real.astype(np.complex128))
    with _clenshaw(Plan(B, device=DEV)) as p:
        g = p.inverse_real(torch.from_numpy(c_sym).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(g, oracle.inverse(B, c_sym).real) < TOL


def test_clenshaw_sampled_B256():
    B = 256
    coef = synth.coefficients(B, "gauss_decay", seed=8999)
    rng = np.random.default_rng(256)
    n = 2 * B
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1)] + [tuple(int(v) for v in rng.integers(0, n, size=3)) for _ in range(6)]
    with _clenshaw(Plan(B, device=DEV)) as p:
        g = p.inverse(torch.from_numpy(coef).to(DEV))
        p.sync()
        got = np.array([g[j, i, k].item() for (i, j, k) in pts])
    prev = oracle.set_threads(8)
    try:
        want = oracle.inverse_points(B, coef, pts)
    finally:
        oracle.set_threads(prev)
    assert synth.rel_l2(got, want) < TOL
