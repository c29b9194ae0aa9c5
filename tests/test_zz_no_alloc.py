"""soft_dwt_forward_noalloc: the forward DWT for callers that cannot allocate
device memory (for example a plug-in whose host application owns the whole
device memory pool, or a pipeline that allocates only at start-up).  It keeps
its tables in a fixed static device array instead of a plan.

Checked through the C ABI against the plan-based soft_dwt_forward on two calls
in a row (different bandwidths, so the second call must not depend on what the
first left in the shared array), with the FP64 tolerance of the other parity
tests.  This file is named to be collected last.
"""

import numpy as np
import pytest
import torch

from paper_1808_00896_gb300 import Plan, capi, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _random_S(B, seed):
    # any complex array in the S layout; the DWT reads only |m|, |m'| < B
    return torch.from_numpy(synth.random_grid(B, seed=seed)).to(DEV)


def test_noalloc_matches_plan_path_two_calls_in_a_row():
    lib = capi.load()
    torch.cuda.set_device(DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    for B, seed in ((64, 11), (23, 12)):
        S = _random_S(B, seed)
        with Plan(B, device=DEV) as p:
            ref = p.dwt_forward(S).cpu().numpy()
        out = torch.full((synth.num_coeffs(B),), complex(float("nan"), float("nan")),
                         dtype=torch.complex128, device=DEV)
        st = lib.soft_dwt_forward_noalloc(B, S.data_ptr(), out.data_ptr(), stream)
        assert st == capi.SOFT_OK, capi.status_string(st)
        torch.cuda.synchronize(DEV)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert synth.rel_l2(got, ref) < TOL


def test_noalloc_rejects_bandwidth_above_limit():
    lib = capi.load()
    B = 257
    S = torch.zeros(8, dtype=torch.complex128, device=DEV)
    c = torch.zeros(8, dtype=torch.complex128, device=DEV)
    st = lib.soft_dwt_forward_noalloc(B, S.data_ptr(), c.data_ptr(), None)
    assert st == capi.SOFT_ERR_UNSUPPORTED
    assert "static scratch limit" in lib.soft_last_error().decode()
    assert lib.soft_dwt_forward_noalloc(0, S.data_ptr(), c.data_ptr(), None) == capi.SOFT_ERR_INVALID_ARG
