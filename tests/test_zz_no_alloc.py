"""soft_dwt_forward_noalloc: the forward DWT for callers that cannot allocate
device memory (for example a plug-in whose host application owns the whole
device memory pool, or a pipeline that allocates only at start-up).  It keeps
its tables in a fixed static device array instead of a plan, and computes
the seeds and recurrence coefficients on the fly instead of loading a plan's
tables.

Checked through the C ABI against the oracle (the DWT of the oracle's own
2-D DFT of a grid equals the oracle's forward transform of that grid), at
B = 1, 2, 8, 23, 64 in full and at the documented limit B = 256 on sampled
order pairs and in full against the plan-based soft_dwt_forward; on calls in a
row of different bandwidths on one stream (each call must not depend on what
the previous one left in the shared array).  This file is named to be
collected last.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_1808_00896_gb300 import Plan, capi, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    prev = oracle.set_threads(max(1, len(__import__("os").sched_getaffinity(0))))
    yield
    oracle.set_threads(prev)


def _oracle_S(B, grid):
    """S[j][m mod 2B][m' mod 2B]: the oracle's unnormalised exp(+i) 2-D DFT of each beta slice."""
    return oracle.dft2_slices(grid, +1)


def _call(lib, B, S_dev, stream):
    out = torch.full((synth.num_coeffs(B),), complex(float("nan"), float("nan")),
                     dtype=torch.complex128, device=DEV)
    st = lib.soft_dwt_forward_noalloc(B, S_dev.data_ptr(), out.data_ptr(), stream)
    assert st == capi.SOFT_OK, (capi.status_string(st), lib.soft_last_error())
    return out


def test_noalloc_matches_oracle_calls_in_a_row():
    lib = capi.load()
    torch.cuda.set_device(DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    cases = []
    for B, seed in ((64, 11), (23, 12), (1, 13), (2, 14), (8, 15)):
        grid = synth.random_grid(B, seed=seed)
        cases.append((B, torch.from_numpy(_oracle_S(B, grid)).to(DEV), oracle.forward(B, grid)))
    # all calls queued back to back on one stream before any synchronisation
    outs = [_call(lib, B, S, stream) for B, S, _ in cases]
    torch.cuda.synchronize(DEV)
    for (B, _, want), out in zip(cases, outs):
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), B
        assert synth.rel_l2(got, want) < TOL, B


def test_noalloc_at_its_limit_alternating_with_a_small_bandwidth():
    """B = 256 (2B = 512, the largest tile shape the entry point takes), then
    B = 8, then B = 256 again on one stream: sampled order pairs of every
    length against the oracle, the whole vector against the plan path, and
    the two B = 256 calls identical."""
    lib = capi.load()
    torch.cuda.set_device(DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    B = 256
    grid = synth.random_grid(B, seed=4256)
    S = torch.from_numpy(_oracle_S(B, grid)).to(DEV)
    g8 = synth.random_grid(8, seed=4008)
    S8 = torch.from_numpy(_oracle_S(8, g8)).to(DEV)
    a = _call(lib, B, S, stream)
    b = _call(lib, 8, S8, stream)
    c = _call(lib, B, S, stream)
    torch.cuda.synchronize(DEV)
    with Plan(B, device=DEV) as p:
        ref = p.dwt_forward(S)
        p.sync()
    a_h, c_h = a.cpu().numpy(), c.cpu().numpy()
    assert np.isfinite(a_h).all()
    assert np.array_equal(a_h, c_h)
    assert synth.rel_l2(a_h, ref.cpu().numpy()) < TOL
    assert synth.rel_l2(b.cpu().numpy(), oracle.forward(8, g8)) < TOL
    rng = np.random.default_rng(256)
    pairs = [(0, 0), (B - 1, B - 1), (1 - B, 0), (B // 2, -(B // 3))]
    pairs += [tuple(int(v) for v in rng.integers(1 - B, B, size=2)) for _ in range(4)]
    want = np.concatenate(oracle.forward_pairs(B, grid, pairs))
    got = []
    for m, mp in pairs:
        l0 = max(abs(m), abs(mp))
        o = capi.soft_coef_index(B, l0, m, mp)
        got.append(a_h[o:o + B - l0])
    assert synth.rel_l2(np.concatenate(got), want) < TOL


def test_noalloc_rejects_bandwidth_above_limit():
    lib = capi.load()
    B = 257
    S = torch.zeros(8, dtype=torch.complex128, device=DEV)
    c = torch.zeros(8, dtype=torch.complex128, device=DEV)
    st = lib.soft_dwt_forward_noalloc(B, S.data_ptr(), c.data_ptr(), None)
    assert st == capi.SOFT_ERR_UNSUPPORTED
    assert "static scratch limit" in lib.soft_last_error().decode()
    assert lib.soft_dwt_forward_noalloc(0, S.data_ptr(), c.data_ptr(), None) == capi.SOFT_ERR_INVALID_ARG
