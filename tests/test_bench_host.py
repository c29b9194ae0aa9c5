"""Host-side pieces of bench.py, on the CPU: the algorithmic work the roofline
divides by, counted by brute force over the clusters, and the workload table.
"""
import os

import pytest

import bench


def _clusters(B):
    """Representatives m >= m' >= 0 and their partner counts (1, 4 or 8), as
    the symmetry relations of Eq. (Wigner_symmetries) group the order pairs."""
    for m in range(B):
        for mp in range(m + 1):
            yield m, mp, 1 if m == mp == 0 else 4 if (mp == 0 or m == mp) else 8


@pytest.mark.parametrize("B", [1, 2, 3, 8, 17, 64])
def test_dwt_flops_by_brute_force(B):
    fl = bench.dwt_flops(B)
    n = 2 * B
    # every order pair (m, m') with |m|, |m'| < B has the run l = max(|m|,|m'|) .. B-1
    runs = sum(B - max(abs(m), abs(mp)) for m in range(1 - B, B) for mp in range(1 - B, B))
    assert runs == B * (4 * B * B - 1) // 3
    # each coefficient: 2B real-weighted complex terms, one FMA (2 flops) per real part
    assert fl["contraction"] == runs * n * 2 * 2
    # the clusters cover every order pair once
    assert sum(np_ for _, _, np_ in _clusters(B)) == (2 * B - 1) ** 2
    # one Wigner-d column block per cluster: B - m degrees x 2B samples, 2 FMAs each
    entries = sum((B - m) * n for m, _, _ in _clusters(B))
    assert fl["t_entries"] == entries
    assert fl["recurrence"] == 4 * entries


def test_dwt_flops_at_the_benchmark_size():
    fl = bench.dwt_flops(64)
    assert fl["contraction"] + fl["recurrence"] == 202_375_168  # the bench line's algorithmic_flops_per_launch


def test_workloads_are_well_formed():
    for name, (B, mode, kind, desc) in bench.WORKLOADS.items():
        assert 1 <= B <= 512 and desc
        assert mode in ("fp64", "fp64_real", "fp64_clenshaw", "fp64_tc", "fp64_tc_real", "bf16x3", "tf32"), name
        assert kind in ("uniform", "gauss_decay"), name
        if mode.endswith("_real"):  # the real entry points need power-of-two 2B
            assert (2 * B) & (2 * B - 1) == 0, name
    assert bench.WORKLOADS["b256"][:2] == (256, "fp64")  # the default workload


def test_traffic_entries_name_existing_sources():
    for (kernel, B), (nbytes, src, sha) in bench.TRAFFIC.items():
        path = os.path.join(bench.ROOT, "paper_1808_00896_gb300", "csrc", src)
        assert os.path.exists(path), src
        assert kernel in open(path).read(), (kernel, src)
        assert nbytes > 16 * (2 * B) ** 3, "a forward DWT reads all of S at least once"
        assert len(sha) == 16


def test_source_sha_ignores_comments_but_not_code(tmp_path, monkeypatch):
    """A recorded traffic figure stays valid across comment edits of its
    kernel's source and is voided by any change of the code."""
    d = tmp_path / "paper_1808_00896_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    versions = {
        "base": "// header\nint f(int a) {  /* old */\n  return a + 1;\n}\n",
        "comments": "// a longer header\n// over two lines\n\nint f(int a) {  /* new\n  text */\n  return a + 1;  // sum\n}\n",
        "code": "// header\nint f(int a) {  /* old */\n  return a + 2;\n}\n",
    }
    sha = {}
    for k, text in versions.items():
        (d / "k.cu").write_text(text)
        sha[k] = bench.kernel_source_sha("k.cu")
    assert sha["base"] == sha["comments"]
    assert sha["base"] != sha["code"]


@pytest.mark.parametrize("B", [1, 2, 3, 8, 64, 512])
def test_sampled_pairs_and_points_are_in_range(B):
    pairs = bench.sample_pairs(B, seed=B)
    assert len(pairs) == len(set(pairs)) == min(16, (2 * B - 1) ** 2)
    assert all(max(abs(m), abs(mp)) < B for m, mp in pairs)
    if B >= 8:  # runs of every length band, the longest and the shortest included
        l0s = {max(abs(m), abs(mp)) for m, mp in pairs}
        assert 0 in l0s and B - 1 in l0s and len(l0s) >= 8
    pts = bench.sample_points(B, seed=B)
    assert all(0 <= v < 2 * B for p in pts for v in p)


def test_oracle_ref_indexing_against_the_oracle_itself():
    """OracleRef gathers the sampled runs and points from full output arrays;
    fed the oracle's own full transforms it must report rounding-level errors."""
    import numpy as np
    import torch

    import oracle
    from paper_1808_00896_gb300 import build as build_mod
    from paper_1808_00896_gb300 import synth
    build_mod.build()  # OracleRef reads run offsets through the library's host-only soft_coef_index
    B = 8
    coef = synth.coefficients(B, "gauss_decay", seed=3)
    grid = oracle.inverse(B, coef)
    ref = bench.OracleRef(B, grid, coef, seed=4, threads=2)
    err = ref.errors(torch.from_numpy(oracle.forward(B, grid)), torch.from_numpy(grid))
    assert err["forward"] < 1e-13 and err["inverse"] < 1e-13
    # a wrong run is seen
    bad = oracle.forward(B, grid)
    bad[ref.coef_idx[0]] += 1.0
    assert ref.errors(torch.from_numpy(bad), torch.from_numpy(grid))["forward"] > 1e-3


def test_every_single_workload_exceeds_l2_per_pass():
    """The timing rule: between timed steps the inputs are not L2-resident.
    For every single-transform workload the rotated input sets span at least
    twice the L2, or one set alone exceeds it, and the config says which."""
    import types
    for name, (B, dtype, kind, _) in bench.WORKLOADS.items():
        if name in bench.BATCHED:
            continue
        c = bench.workload_config(types.SimpleNamespace(workload=name), B, dtype, kind, 1)
        n = 2 * B
        set_bytes = (8 if "real" in dtype else 16) * n ** 3 + 16 * (B * (4 * B * B - 1) // 3)
        R = c["inputs_rotated"]
        assert R * set_bytes >= 2 * bench.L2_BYTES or (R == 1 and set_bytes > bench.L2_BYTES), name
        assert ("single input larger than L2" in c["l2"]) == (R == 1), name
