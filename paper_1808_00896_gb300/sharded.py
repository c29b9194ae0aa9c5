"""One SO(3) transform sharded over several GPUs (one process per GPU).

The two steps of the fast transform (Sec. 2.4) want the data split two ways:
the 2-D FFT of a beta slice needs every order pair (m, m') of that slice, the
DWT of a symmetry cluster (Sec. 3) needs every beta slice of its partners'
order pairs.  Rank r of R therefore owns

* the beta slices [slice_range(B, R, r)) of the grid, and
* the symmetry clusters ``cluster_shard(B, R, r)`` (balanced by work),

and one all-to-all between the steps moves the S columns: in the forward,
each rank sends every other rank that rank's partner columns over its own
slices; the inverse runs the steps backwards.  Every step of the arithmetic
runs in the library's kernels (slice FFTs, cluster-subset DWT / iDWT, column
gather / scatter); this module only lays out the exchange and calls the
collective (``torch.distributed.all_to_all``, NCCL between GPUs).

Coefficients stay in the full coefficient layout: a rank's forward writes its
own clusters' runs, and its inverse reads only those.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi
from .api import Plan, _check_tensor, _stream_ptr


def slice_range(B: int, world: int, rank: int) -> tuple[int, int]:
    """Beta slices [j0, j1) of rank `rank` of `world`: contiguous, sizes differing by at most one."""
    n = 2 * B
    return rank * n // world, (rank + 1) * n // world


def cluster_shard(B: int, world: int, rank: int) -> np.ndarray:
    """Representatives (m, m') of the clusters rank `rank` owns (soft_cluster_shard), int32 (count, 2)."""
    out = np.zeros(B * (B + 1), dtype=np.int32)
    cnt = np.zeros(1, dtype=np.int32)
    capi.check(capi.load().soft_cluster_shard(B, world, rank, out.ctypes.data, cnt.ctypes.data), "soft_cluster_shard")
    return out[:2 * int(cnt[0])].reshape(-1, 2).copy()


def cluster_columns(reps: np.ndarray) -> np.ndarray:
    """Order pairs of the clusters' partners, the S columns they use (soft_cluster_columns), int32 (npairs, 2)."""
    reps = np.ascontiguousarray(reps, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(16 * max(1, len(reps)), dtype=np.int32)
    k = capi.load().soft_cluster_columns(len(reps), reps.ctypes.data, out.ctypes.data)
    if k < 0:
        raise ValueError("bad cluster representatives")
    return out[:2 * k].reshape(-1, 2).copy()


def exchange_shapes(B: int, world: int, rank: int, forward: bool) -> tuple[list, list]:
    """(send shapes, receive shapes) of rank `rank`'s buffers, one per rank,
    each (slices, columns) complex values.  Forward: rank r sends rank d the
    columns of d's clusters over r's slices.  Inverse: rank r sends rank d the
    columns of r's clusters over d's slices."""
    ranges = [slice_range(B, world, r) for r in range(world)]
    ncols = [len(cluster_columns(cluster_shard(B, world, r))) for r in range(world)]
    j0, j1 = ranges[rank]
    if forward:
        sends = [(j1 - j0, ncols[d]) for d in range(world)]
        recvs = [(b - a, ncols[rank]) for (a, b) in ranges]
    else:
        sends = [(b - a, ncols[rank]) for (a, b) in ranges]
        recvs = [(j1 - j0, ncols[s]) for s in range(world)]
    return sends, recvs


def all_to_all(sends: list[torch.Tensor], recvs: list[torch.Tensor], group=None) -> None:
    """The exchange: rank r's sends[d] lands in rank d's recvs[r]
    (torch.distributed point-to-point operations, posted together: one
    send and one receive per peer; NCCL groups them into one exchange, and
    gloo, which has no all-to-all of tensor lists, runs them as well).  The
    rank's own block is copied locally."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    ops = []
    for peer, (snd, rcv) in enumerate(zip(sends, recvs)):
        if peer == rank:
            rcv.copy_(snd)
            continue
        gpeer = dist.get_global_rank(group, peer) if group is not None else peer
        if snd.numel():
            ops.append(dist.P2POp(dist.isend, snd.contiguous(), gpeer, group))
        if rcv.numel():
            ops.append(dist.P2POp(dist.irecv, rcv, gpeer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class ShardedTransform:
    """Rank `rank`'s share of one forward / inverse transform of bandwidth B
    sharded over `world` ranks (FP64 or FP64-TC plans, power-of-two 2B).

    ``forward`` / ``inverse`` run the whole sharded step with ``exchange``
    (default: torch.distributed.all_to_all).  The phase methods
    (``forward_send`` / ``forward_finish``, ``inverse_send`` /
    ``inverse_finish``) expose the two halves around the exchange."""

    def __init__(self, B: int, world: int, rank: int, dtype: str = "fp64", device=None, exchange=None):
        if not 0 <= rank < world:
            raise ValueError("rank must be in [0, world)")
        self.B, self.world, self.rank = int(B), int(world), int(rank)
        self.n = 2 * self.B
        self.plan = Plan(self.B, dtype, device=device)
        self.device = self.plan.device
        self.j0, self.j1 = slice_range(self.B, world, rank)
        self.ranges = [slice_range(self.B, world, r) for r in range(world)]
        self.reps = [cluster_shard(self.B, world, r) for r in range(world)]
        self.cols = [cluster_columns(rp) for rp in self.reps]
        self.exchange = exchange or all_to_all
        n = self.n
        self.S = torch.empty(n ** 3, dtype=torch.complex128, device=self.device)  # full-layout S workspace

    def close(self) -> None:
        self.plan.close()

    # -- helpers ---------------------------------------------------------------
    def _lib(self):
        return capi.load()

    def _s(self, stream=None) -> int:
        return _stream_ptr(self.device, stream)

    def _slice_ptr(self, j: int) -> int:
        return self.S.data_ptr() + 16 * j * self.n * self.n

    def _gather(self, j0: int, j1: int, cols: np.ndarray, stream=None) -> torch.Tensor:
        out = torch.empty((j1 - j0, len(cols)), dtype=torch.complex128, device=self.device)
        if out.numel() == 0:
            return out
        c = np.ascontiguousarray(cols, dtype=np.int32)
        capi.check(self._lib().soft_gather_columns(self.plan.handle, self.S.data_ptr(), j0, j1 - j0, c.ctypes.data,
                                                   len(c), out.data_ptr(), self._s(stream)), "soft_gather_columns")
        return out

    def _scatter(self, buf: torch.Tensor, j0: int, j1: int, cols: np.ndarray, stream=None) -> None:
        if buf.numel() == 0:
            return
        c = np.ascontiguousarray(cols, dtype=np.int32)
        capi.check(self._lib().soft_scatter_columns(self.plan.handle, buf.data_ptr(), j0, j1 - j0, c.ctypes.data,
                                                    len(c), self.S.data_ptr(), self._s(stream)),
                   "soft_scatter_columns")

    def _empty_recvs(self, forward: bool) -> list[torch.Tensor]:
        _, shapes = exchange_shapes(self.B, self.world, self.rank, forward)
        return [torch.empty(sh, dtype=torch.complex128, device=self.device) for sh in shapes]

    # -- forward -----------------------------------------------------------------
    def forward_send(self, grid_local: torch.Tensor, stream=None) -> list[torch.Tensor]:
        """Slice FFTs of this rank's slices into S, then one buffer per rank d:
        d's partner columns over this rank's slices."""
        _check_tensor(grid_local, (self.j1 - self.j0) * self.n ** 2, self.device, "grid_local")
        if self.j1 > self.j0:
            capi.check(self._lib().soft_slice_fft(self.plan.handle, grid_local.data_ptr(), self._slice_ptr(self.j0),
                                                  1, self.j0, self.j1 - self.j0, self._s(stream)), "soft_slice_fft")
        return [self._gather(self.j0, self.j1, self.cols[d], stream) for d in range(self.world)]

    def forward_finish(self, recvs: list[torch.Tensor], coef: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Every rank's slices of this rank's partner columns into S, then the
        DWT of this rank's clusters (writes their coefficient runs)."""
        coef = self.plan.empty_coef() if coef is None else coef
        _check_tensor(coef, self.plan.ncoef, self.device, "coef")
        for (j0, j1), buf in zip(self.ranges, recvs):
            self._scatter(buf, j0, j1, self.cols[self.rank], stream)
        rp = np.ascontiguousarray(self.reps[self.rank], dtype=np.int32)
        capi.check(self._lib().soft_dwt_forward_clusters(self.plan.handle, self.S.data_ptr(), coef.data_ptr(),
                                                         rp.ctypes.data, len(rp), self._s(stream)),
                   "soft_dwt_forward_clusters")
        return coef

    def forward(self, grid_local: torch.Tensor, coef: torch.Tensor | None = None) -> torch.Tensor:
        sends = self.forward_send(grid_local)
        recvs = self._empty_recvs(True)
        self.exchange(sends, recvs)
        return self.forward_finish(recvs, coef)

    # -- inverse -----------------------------------------------------------------
    def inverse_send(self, coef: torch.Tensor, stream=None) -> list[torch.Tensor]:
        """iDWT of this rank's clusters into S (their columns, every slice),
        then one buffer per rank d: this rank's columns over d's slices."""
        _check_tensor(coef, self.plan.ncoef, self.device, "coef")
        rp = np.ascontiguousarray(self.reps[self.rank], dtype=np.int32)
        capi.check(self._lib().soft_dwt_inverse_clusters(self.plan.handle, coef.data_ptr(), self.S.data_ptr(),
                                                         rp.ctypes.data, len(rp), self._s(stream)),
                   "soft_dwt_inverse_clusters")
        return [self._gather(j0, j1, self.cols[self.rank], stream) for (j0, j1) in self.ranges]

    def inverse_finish(self, recvs: list[torch.Tensor], grid_local: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
        """Every rank's columns over this rank's slices into S, then the
        inverse slice FFTs of this rank's slices."""
        ns = self.j1 - self.j0
        grid_local = torch.empty((ns, self.n, self.n), dtype=torch.complex128, device=self.device) \
            if grid_local is None else grid_local
        _check_tensor(grid_local, ns * self.n ** 2, self.device, "grid_local")
        for s, buf in enumerate(recvs):
            self._scatter(buf, self.j0, self.j1, self.cols[s], stream)
        if ns > 0:
            capi.check(self._lib().soft_slice_fft(self.plan.handle, self._slice_ptr(self.j0), grid_local.data_ptr(),
                                                  -1, self.j0, ns, self._s(stream)), "soft_slice_fft")
        return grid_local

    def inverse(self, coef: torch.Tensor, grid_local: torch.Tensor | None = None) -> torch.Tensor:
        sends = self.inverse_send(coef)
        recvs = self._empty_recvs(False)
        self.exchange(sends, recvs)
        return self.inverse_finish(recvs, grid_local)
