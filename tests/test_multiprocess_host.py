"""The multi-process host logic of bench.py on CPU: with one process per GPU
each rank runs its own replica of the workload (the transforms are
independent, so there is no collective on the data path) and the timed region
is combined as the maximum over ranks.  Checked here with world_size 2 on the
gloo backend."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_setup()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    out[rank] = (w, r, lr, bench.max_over_ranks(ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == (2, 0, 0, 15.0)
    assert out[1] == (2, 1, 1, 15.0)


def test_max_over_ranks_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    if dist.is_available() and dist.is_initialized():
        pytest.skip("a process group is active")
    assert bench.max_over_ranks(3.5) == 3.5
