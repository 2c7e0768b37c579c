"""Sharded propagation sweeps (include/pg.h, "Sharded sweeps") on one GPU:
every shard's pack, halo copy and sweep run one after another on the same
device, in the order the ranks of a multi-GPU job run them (the exchange
is a device copy here instead of NCCL send/recv), and the gathered rows
must equal pg_propagate's iterate bit for bit."""
import ctypes

import numpy as np
import pytest
import torch

import pgrec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_11894_gb300 as pg

    return pg


@pytest.mark.parametrize("world,wdtype", [(2, "f32"), (3, "f32"), (2, "u16"), (4, "bf16"), (8, "f32"), (8, "u16")])
def test_shards_on_one_device_equal_pg_propagate(pg, world, wdtype):
    from paper_2404_11894_gb300 import _lib, _ptr, _stream_ptr
    from paper_2404_11894_gb300.dist import ShardLists

    lib = _lib.load()
    sc = pgrec.CLOUD128.with_(width=48, height=48, spp=4)
    rec = pgrec.trace(sc)
    V = pg.Vertices.from_records(rec)
    graph = pg.pg_build_graph(V, sc.k)
    pg.pg_aggregate(graph, V, wdtype)
    L0 = torch.from_numpy(rec["L0"]).cuda()
    T = sc.iters
    ref = pg.pg_propagate(graph, L0, T)
    s = _stream_ptr(None)
    n = graph.n
    y = torch.empty(n + 1, dtype=torch.float32, device="cuda")
    _lib.check(lib.pg_graph_y_from_L(graph.handle, _ptr(L0), _ptr(y), s), "pg_graph_y_from_L")
    handles, lists, z, send = [], [], [], []
    try:
        for p in range(world):
            h = ctypes.c_void_p()
            _lib.check(lib.pg_shard_create(graph.handle, world, p, s, ctypes.byref(h)), "pg_shard_create")
            handles.append(h)
            Lp = ShardLists(lib, h)
            lists.append(Lp)
            zz = [torch.full((Lp.local_len,), float("nan"), device="cuda") for _ in range(2)]
            for t in zz:
                _lib.check(lib.pg_shard_load(h, _ptr(y), _ptr(t), s), "pg_shard_load")
            z.append(zz)
            send.append(torch.empty(max(Lp.n_send, 1), device="cuda"))
        rb = lists[0].row_begin
        assert rb[0] == 0 and rb[-1] == graph.info()["n_active"]
        cur = 0
        for _ in range(T):
            for p in range(world):
                _lib.check(lib.pg_shard_pack(handles[p], _ptr(z[p][cur]), _ptr(send[p]), s), "pg_shard_pack")
            for qd in range(world):  # receiver
                Lq = lists[qd]
                for p in range(world):  # sender
                    if p == qd:
                        continue
                    a, b = int(lists[p].send_begin[qd]), int(lists[p].send_begin[qd + 1])
                    c, d = int(Lq.recv_begin[p]), int(Lq.recv_begin[p + 1])
                    assert b - a == d - c
                    z[qd][cur][Lq.rows + c:Lq.rows + d] = send[p][a:b]
            for p in range(world):
                _lib.check(lib.pg_shard_sweep(handles[p], _ptr(z[p][cur]), _ptr(z[p][1 - cur]), s),
                           "pg_shard_sweep")
            cur = 1 - cur
        for p in range(world):
            a, b = int(rb[p]), int(rb[p + 1])
            y[a:b] = z[p][cur][:b - a]
        L = torch.empty(n, dtype=torch.float32, device="cuda")
        _lib.check(lib.pg_graph_L_from_y(graph.handle, _ptr(y), _ptr(L), s), "pg_graph_L_from_y")
        torch.cuda.synchronize()
        assert torch.equal(L, ref)
        # the halo exchange is a small part of the vector: rows read across slabs
        halo = sum(Lp.n_halo for Lp in lists)
        print(f"\n{world} shards, {wdtype}: halo entries {halo} of {int(rb[-1])} rows")
    finally:
        for h in handles:
            lib.pg_shard_destroy(h)
        graph.close()


def test_sharded_propagator_single_rank(pg):
    """ShardedPropagator with one shard (no process group): the whole sweep
    through the shard path equals pg_propagate."""
    from paper_2404_11894_gb300.dist import ShardedPropagator

    sc = pgrec.CLOUD128.with_(width=40, height=40, spp=4)
    rec = pgrec.trace(sc)
    V = pg.Vertices.from_records(rec)
    graph = pg.pg_build_graph(V, sc.k)
    pg.pg_aggregate(graph, V, "f32")
    L0 = torch.from_numpy(rec["L0"]).cuda()
    ref = pg.pg_propagate(graph, L0, 12)
    sp = ShardedPropagator(graph, 0, 1)
    try:
        L = sp.run(L0, 12)
        torch.cuda.synchronize()
        assert torch.equal(L, ref)
    finally:
        sp.close()
        graph.close()
