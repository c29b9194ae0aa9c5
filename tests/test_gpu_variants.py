"""Every tile-shape variant of the DWT kernels gives the default's result (up
to rounding order), and the autotuner picks and caches one."""
import json

import pytest
import torch

from paper_1808_00896_gb300 import Plan, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_00896_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


# Odd B (129, 257) give 2B samples that 4 threads per output cannot split evenly.
@pytest.mark.parametrize("B,mode", [(16, "fp64"), (100, "fp64"), (129, "fp64"), (200, "fp64"), (257, "fp64"),
                                    (400, "fp64"), (30, "bf16x3"), (200, "tf32")])
def test_variants_agree(B, mode):
    grid = torch.from_numpy(synth.random_grid(B, seed=B)).to(DEV)
    coef = torch.from_numpy(synth.coefficients(B, "gauss_decay", seed=B + 1)).to(DEV)
    tol = 1e-12 if mode == "fp64" else 1e-5
    with Plan(B, mode, device=DEV) as p:
        f0, g0 = p.forward(grid).cpu().numpy(), p.inverse(coef).cpu().numpy()
        for k, ref, fn, x in ((0, f0, p.forward, grid), (1, g0, p.inverse, coef)):
            for v in range(1, p.num_variants(k)):
                p.set_variant(k, v)
                got = fn(x).cpu().numpy()
                p.sync()
                assert synth.rel_l2(got, ref) < tol, (k, v)
            p.set_variant(k, 0)


def test_autotune_caches(tmp_path, monkeypatch):
    path = tmp_path / "tiles.json"
    monkeypatch.setenv("SOFT_TUNE_CACHE", str(path))
    with Plan(64, device=DEV) as p:
        choice = p.tune(reps=2)
        assert 0 <= choice["dwt"] < p.num_variants(0) and 0 <= choice["idwt"] < p.num_variants(1)
    cache = json.loads(path.read_text())
    assert len(cache) == 1 and list(cache.values())[0]["dwt"] == choice["dwt"]
    with Plan(64, device=DEV) as p:  # second plan: served from the cache
        assert p.tune()["dwt"] == choice["dwt"]
