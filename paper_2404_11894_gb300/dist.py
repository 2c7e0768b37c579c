"""Several GPUs, one process per GPU.

Two modes. Replicas: each rank solves its own image (a different seed), with
no data-path collective; only the timing is combined (the job's time is the
maximum over ranks, its work the sum). Shards: the ranks split one graph's
propagation sweeps by Morton slabs of rows and exchange the halo entries of
the sweep vector before every sweep (ShardedPropagator).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def combine_throughput(local_seconds: float, local_units: float, device=None):
    """(max seconds over ranks, total units over ranks); identity on 1 rank."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_seconds), float(local_units)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's independent render."""
    return int(base_seed) + 1000003 * int(rank)


# ----------------------------------------------------------------------------- sharded sweeps
# One shard of the propagation per rank (include/pg.h, "Sharded sweeps"):
# each rank owns a Morton slab of the sweep rows and, before every sweep,
# exchanges with its peers the halo entries their rows read.
import ctypes  # noqa: E402

import numpy as np  # noqa: E402


class ShardLists:
    """A shard's plan as host arrays (pg_shard_get_info / pg_shard_get_lists)."""

    def __init__(self, lib, handle):
        from ._lib import PgShardInfo, check

        info = PgShardInfo()
        check(lib.pg_shard_get_info(handle, ctypes.byref(info)), "pg_shard_get_info")
        self.n_shards, self.shard, self.row_width = info.n_shards, info.shard, info.row_width
        self.row_begin_own, self.row_end_own = info.row_begin, info.row_end
        self.rows = info.row_end - info.row_begin
        self.n_halo, self.local_len, self.n_send = info.n_halo, info.local_len, info.n_send
        P = info.n_shards
        self.row_begin = np.zeros(P + 1, np.int64)
        self.recv_begin = np.zeros(P + 1, np.int64)
        self.send_begin = np.zeros(P + 1, np.int64)
        self.halo = np.zeros(max(self.n_halo, 1), np.int32)
        self.send_idx = np.zeros(max(self.n_send, 1), np.int32)
        self.local_col = np.zeros(max(self.rows * self.row_width, 1), np.int32)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        check(lib.pg_shard_get_lists(handle, ptr(self.row_begin), ptr(self.recv_begin), ptr(self.send_begin),
                                     ptr(self.halo), ptr(self.send_idx), ptr(self.local_col)), "pg_shard_get_lists")
        self.halo = self.halo[:self.n_halo]
        self.send_idx = self.send_idx[:self.n_send]
        self.local_col = self.local_col[:self.rows * self.row_width].reshape(self.rows, self.row_width)


def shard_plan_host(col: np.ndarray, zero_slot: int, n_shards: int, shard: int) -> ShardLists:
    """The partition of a host column table (rows x row width) without a
    device (pg_shard_create_host)."""
    from ._lib import check, load

    lib = load()
    col = np.ascontiguousarray(col, np.int32)
    h = ctypes.c_void_p()
    check(lib.pg_shard_create_host(col.ctypes.data_as(ctypes.c_void_p), col.shape[0], col.shape[1], zero_slot,
                                   n_shards, shard, ctypes.byref(h)), "pg_shard_create_host")
    try:
        return ShardLists(lib, h)
    finally:
        lib.pg_shard_destroy(h)


def exchange_halo(send: torch.Tensor, lists: ShardLists, z: torch.Tensor, group=None):
    """Peer-to-peer halo exchange of one sweep: the segment of ``send`` for
    each peer goes to it, and each peer's segment lands in its part of the
    halo of ``z`` (own rows first, then the halo). Works on CPU tensors with
    gloo and on CUDA tensors with NCCL."""
    ops = []
    me = lists.shard
    for q in range(lists.n_shards):
        if q == me:
            continue
        a, b = int(lists.send_begin[q]), int(lists.send_begin[q + 1])
        if b > a:
            ops.append(dist.P2POp(dist.isend, send[a:b], q, group))
        a, b = int(lists.recv_begin[q]), int(lists.recv_begin[q + 1])
        if b > a:
            ops.append(dist.P2POp(dist.irecv, z[lists.rows + a:lists.rows + b], q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class ShardedPropagator:
    """pg_propagate split over the ranks of a process group, one shard per
    rank and GPU: T sweeps with one halo exchange before each, then the
    shards' rows gathered into L+ (the same bits as pg_propagate)."""

    def __init__(self, graph, rank: int, world: int, group=None):
        from ._lib import check, load

        self.lib = load()
        self.graph, self.rank, self.world, self.group = graph, rank, world, group
        self.handle = ctypes.c_void_p()
        check(self.lib.pg_shard_create(graph.handle, world, rank, None, ctypes.byref(self.handle)),
              "pg_shard_create")
        self.lists = ShardLists(self.lib, self.handle)
        dev = torch.device("cuda")
        self.z = [torch.empty(self.lists.local_len, dtype=torch.float32, device=dev) for _ in range(2)]
        self.send = torch.empty(max(self.lists.n_send, 1), dtype=torch.float32, device=dev)

    def run(self, L0: torch.Tensor, iters: int) -> torch.Tensor:
        from . import _ptr, _stream_ptr
        from ._lib import check

        n = self.graph.n
        y = torch.empty(n + 1, dtype=torch.float32, device="cuda")
        s = _stream_ptr(None)
        check(self.lib.pg_graph_y_from_L(self.graph.handle, _ptr(L0), _ptr(y), s), "pg_graph_y_from_L")
        for z in self.z:
            check(self.lib.pg_shard_load(self.handle, _ptr(y), _ptr(z), s), "pg_shard_load")
        cur = 0
        for _ in range(iters):
            z_in, z_out = self.z[cur], self.z[1 - cur]
            check(self.lib.pg_shard_pack(self.handle, _ptr(z_in), _ptr(self.send), s), "pg_shard_pack")
            exchange_halo(self.send, self.lists, z_in, self.group)
            check(self.lib.pg_shard_sweep(self.handle, _ptr(z_in), _ptr(z_out), s), "pg_shard_sweep")
            cur = 1 - cur
        # the shards' own rows into the sweep vector on every rank
        width = int(max(self.lists.row_begin[q + 1] - self.lists.row_begin[q] for q in range(self.world)))
        mine = torch.zeros(max(width, 1), dtype=torch.float32, device="cuda")
        mine[:self.lists.rows] = self.z[cur][:self.lists.rows]
        parts = [torch.empty_like(mine) for _ in range(self.world)] if self.world > 1 else [mine]
        if self.world > 1:
            dist.all_gather(parts, mine, group=self.group)
        for q in range(self.world):
            a, b = int(self.lists.row_begin[q]), int(self.lists.row_begin[q + 1])
            y[a:b] = parts[q][:b - a]
        L = torch.empty(n, dtype=torch.float32, device="cuda")
        check(self.lib.pg_graph_L_from_y(self.graph.handle, _ptr(y), _ptr(L), s), "pg_graph_L_from_y")
        return L

    def close(self):
        if self.handle:
            self.lib.pg_shard_destroy(self.handle)
            self.handle = ctypes.c_void_p()
