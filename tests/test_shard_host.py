"""Host side of the sharded transform (one transform over several GPUs): the
cluster partition (every symmetry cluster on exactly one rank, balanced by
work), the S columns each rank's clusters use (every order pair exactly
once), the beta-slice ranges, and the exchange itself between world_size 2
CPU processes on gloo: every block lands where the layout says."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1808_00896_gb300 import sharded


def _work(B, m, mp_):
    np_ = 1 if m == mp_ == 0 else 4 if (mp_ == 0 or m == mp_) else 8
    return (B - m) * 16 + np_


@pytest.mark.parametrize("B,world", [(1, 1), (2, 3), (8, 2), (16, 3), (64, 4), (128, 8), (5, 7)])
def test_cluster_partition(B, world):
    seen = []
    loads = []
    for r in range(world):
        reps = sharded.cluster_shard(B, world, r)
        assert np.all(reps[:, 1] >= 0) and np.all(reps[:, 1] <= reps[:, 0]) and np.all(reps[:, 0] < B)
        seen += [tuple(x) for x in reps]
        loads.append(sum(_work(B, int(m), int(p)) for m, p in reps))
    assert sorted(seen) == sorted((m, p) for m in range(B) for p in range(m + 1))
    # greedy longest-first: no rank exceeds another by more than the largest cluster
    assert max(loads) - min(loads) <= _work(B, 0, 0) + 8


@pytest.mark.parametrize("B,world", [(1, 1), (4, 2), (16, 3), (33, 5)])
def test_columns_cover_every_order_pair_once(B, world):
    cols = np.concatenate([sharded.cluster_columns(sharded.cluster_shard(B, world, r)) for r in range(world)])
    assert sorted(map(tuple, cols)) == sorted((m, p) for m in range(1 - B, B) for p in range(1 - B, B))


@pytest.mark.parametrize("B,world", [(1, 1), (1, 2), (8, 3), (256, 8)])
def test_slice_ranges_partition_the_slices(B, world):
    rs = [sharded.slice_range(B, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == 2 * B
    assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
    assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def _mark(src, dst, shape):
    js, c = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    return torch.from_numpy((1000 * src + 100 * dst + 10 * js + c + 1j * (src - dst)).astype(np.complex128))


def _exchange_rank(rank, world, port, B, forward, errs):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sends_sh, recvs_sh = sharded.exchange_shapes(B, world, rank, forward)
        sends = [_mark(rank, d, sh) for d, sh in enumerate(sends_sh)]
        recvs = [torch.empty(sh, dtype=torch.complex128) for sh in recvs_sh]
        sharded.all_to_all(sends, recvs)
        for s, buf in enumerate(recvs):
            if not torch.equal(buf, _mark(s, rank, recvs_sh[s])):
                errs.put(f"rank {rank} got a wrong block from {s}")
    except Exception as e:  # reported to the parent
        errs.put(f"rank {rank}: {e!r}")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("forward", [True, False])
def test_exchange_on_gloo(forward):
    world, B = 2, 8
    ctx = mp.get_context("spawn")
    errs = ctx.Queue()
    port = 29600 + (1 if forward else 2)
    procs = [ctx.Process(target=_exchange_rank, args=(r, world, port, B, forward, errs)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    msgs = []
    while not errs.empty():
        msgs.append(errs.get())
    assert not msgs, msgs
    # the shapes agree pairwise: what r sends d is what d receives from r
    for r in range(world):
        s_sh, _ = sharded.exchange_shapes(B, world, r, forward)
        for d in range(world):
            _, r_sh = sharded.exchange_shapes(B, world, d, forward)
            assert s_sh[d] == r_sh[r]
