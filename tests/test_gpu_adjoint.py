"""GPU adjoints and autograd: soft_forward_adjoint / soft_inverse_adjoint vs
the oracle's adjoints, the dot test, central finite differences of a scalar
objective (step 1e-6, FP64) at B = 8 and 16, and torch.autograd.gradcheck."""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, soft_forward, soft_inverse, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
BOUND = {"fp64": 1e-10, "bf16x3": 5e-5, "tf32": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("mode", ["fp64", "bf16x3", "tf32"])
@pytest.mark.parametrize("B", [1, 3, 8, 16, 64])
def test_adjoint_parity(mode, B):
    c = synth.coefficients(B, "uniform", seed=11000 + B)
    x = synth.random_grid(B, seed=12000 + B)
    with Plan(B, mode, device=DEV) as p:
        fa = p.forward_adjoint(torch.from_numpy(c).to(DEV)).cpu().numpy()
        ia = p.inverse_adjoint(torch.from_numpy(x).to(DEV)).cpu().numpy()
        p.sync()
    assert synth.rel_l2(fa, oracle.forward_adjoint(B, c)) < BOUND[mode]
    assert synth.rel_l2(ia, oracle.inverse_adjoint(B, x)) < BOUND[mode]


@pytest.mark.parametrize("B", [4, 32])
def test_dot_test_on_gpu(B):
    c = torch.from_numpy(synth.coefficients(B, "uniform", seed=13000 + B)).to(DEV)
    x = torch.from_numpy(synth.random_grid(B, seed=14000 + B)).to(DEV)
    with Plan(B, device=DEV) as p:
        lhs = torch.vdot(p.forward(x), c).item()
        rhs = torch.vdot(x.reshape(-1), p.forward_adjoint(c).reshape(-1)).item()
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
        lhs = torch.vdot(p.inverse(c).reshape(-1), x.reshape(-1)).item()
        rhs = torch.vdot(c, p.inverse_adjoint(x)).item()
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("B", [8, 16])
def test_central_finite_differences(B):
    """L(x) = Re <c, F x>: the autograd gradient against (L(x+hv) - L(x-hv)) / 2h."""
    h = 1e-6
    rng = np.random.default_rng(B)
    c = torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=15000 + B)).to(DEV)
    x0 = torch.from_numpy(synth.random_grid(B, seed=16000 + B)).to(DEV)
    v = torch.from_numpy(synth.random_grid(B, seed=17000 + B)).to(DEV)
    with Plan(B, device=DEV) as p:
        def L(x):
            return torch.vdot(c, soft_forward(x, p)).real

        x = x0.clone().requires_grad_(True)
        L(x).backward()
        ana = torch.vdot(x.grad.reshape(-1), v.reshape(-1)).real.item()
        fd = ((L(x0 + h * v) - L(x0 - h * v)) / (2 * h)).item()
        assert abs(ana - fd) < 1e-6 * max(1.0, abs(ana))

        y = torch.from_numpy(synth.random_grid(B, seed=18000 + B)).to(DEV)
        u = torch.from_numpy(synth.coefficients(B, "uniform", seed=19000 + B)).to(DEV)

        def M(cf):
            return torch.vdot(y.reshape(-1), soft_inverse(cf, p).reshape(-1)).real

        cf = c.clone().requires_grad_(True)
        M(cf).backward()
        ana = torch.vdot(cf.grad, u).real.item()
        fd = ((M(c + h * u) - M(c - h * u)) / (2 * h)).item()
        assert abs(ana - fd) < 1e-6 * max(1.0, abs(ana))
    assert rng is not None


def test_gradcheck_small():
    B = 2
    with Plan(B, device=DEV) as p:
        x = torch.from_numpy(synth.random_grid(B, seed=20000)).to(DEV).requires_grad_(True)
        assert torch.autograd.gradcheck(lambda t: soft_forward(t, p), (x,), eps=1e-6, atol=1e-7)
        c = torch.from_numpy(synth.coefficients(B, "uniform", seed=20001)).to(DEV).requires_grad_(True)
        assert torch.autograd.gradcheck(lambda t: soft_inverse(t, p), (c,), eps=1e-6, atol=1e-7)
