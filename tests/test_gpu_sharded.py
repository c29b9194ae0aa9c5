"""GPU: one transform sharded over R ranks, the ranks emulated in one process
on one GPU (each rank's kernels run on their own data; the exchange between
the two halves of each step is done by copying the blocks, since ranks whose
kernels wait on one another may not share a GPU).  The sharded forward and
inverse equal the unsharded transforms bit for bit (every slice FFT and every
cluster's DWT is the same computation), and the oracle to the FP64 bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, synth
from paper_1808_00896_gb300.sharded import ShardedTransform

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _route(all_sends):
    """recvs[d][r] = sends[r][d]: what the all-to-all delivers."""
    R = len(all_sends)
    return [[all_sends[r][d] for r in range(R)] for d in range(R)]


@pytest.mark.parametrize("B,R,mode", [(8, 2, "fp64"), (16, 3, "fp64"), (32, 4, "fp64"), (16, 2, "fp64_tc"),
                                      (1, 2, "fp64"), (64, 5, "fp64")])
def test_sharded_equals_unsharded(B, R, mode):
    n = 2 * B
    grid = torch.from_numpy(synth.random_grid(B, seed=9100 + B)).to(DEV)
    coef = torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=9200 + B)).to(DEV)
    ranks = [ShardedTransform(B, R, r, mode, device=DEV, exchange=lambda s, r: None) for r in range(R)]
    try:
        # forward: every rank's first half, the exchange, every rank's second half
        sends = [t.forward_send(grid[t.j0:t.j1].contiguous()) for t in ranks]
        coef_out = torch.full((synth.num_coeffs(B),), complex(float("nan"), float("nan")),
                              dtype=torch.complex128, device=DEV)
        for t, recvs in zip(ranks, _route(sends)):
            t.forward_finish(recvs, coef_out)  # disjoint runs of one vector
        # inverse
        sends = [t.inverse_send(coef) for t in ranks]
        grid_out = torch.cat([t.inverse_finish(recvs) for t, recvs in zip(ranks, _route(sends))])
        torch.cuda.synchronize(DEV)
        with Plan(B, mode, device=DEV) as p:
            f_ref = p.forward(grid)
            g_ref = p.inverse(coef)
            p.sync()
        assert torch.isfinite(coef_out.real).all()
        assert torch.equal(coef_out, f_ref)
        assert torch.equal(grid_out.reshape(-1), g_ref.reshape(-1))
        g_np = grid.cpu().numpy()
        assert synth.rel_l2(coef_out.cpu().numpy(), oracle.forward(B, g_np)) < 1e-10
        assert synth.rel_l2(grid_out.cpu().numpy(), oracle.inverse(B, coef.cpu().numpy())) < 1e-10
    finally:
        for t in ranks:
            t.close()
