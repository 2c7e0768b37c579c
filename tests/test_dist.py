"""The multi-rank bookkeeping of bench.py with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2404_11894_gb300.dist import combine_throughput, rank_seed

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = combine_throughput(1.0 + rank, 10.0 * (rank + 1))
    dist.barrier()
    q.put((rank, t, u, rank_seed(7, rank)))
    dist.destroy_process_group()


def test_two_ranks_max_time_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [2.0, 2.0]       # max over ranks
    assert [o[2] for o in out] == [30.0, 30.0]     # sum over ranks
    assert out[0][3] != out[1][3]                   # independent renders


def test_single_process_identity():
    from paper_2404_11894_gb300.dist import combine_throughput

    assert combine_throughput(3.0, 5.0) == (3.0, 5.0)


# ----------------------------------------------------------------------------- sharded sweeps (CPU)
def _sweep_problem(n_rows=3000, kp=8, seed=3):
    """A sweep matrix shaped like the path graph's: rows in Morton order read
    mostly nearby rows (neighbours) and some far ones (continuation edges),
    with empty entries pointing at the zero slot."""
    import numpy as np

    rng = np.random.default_rng(seed)
    zero = n_rows
    near = np.clip(np.arange(n_rows)[:, None] + rng.integers(-40, 40, (n_rows, kp)), 0, n_rows - 1)
    far = rng.integers(0, n_rows, (n_rows, kp))
    col = np.where(rng.uniform(size=(n_rows, kp)) < 0.2, far, near)
    col = np.where(rng.uniform(size=(n_rows, kp)) < 0.1, zero, col).astype(np.int32)
    W = rng.uniform(0, 0.1, (n_rows, kp)).astype(np.float32)
    b = rng.uniform(0, 1, n_rows).astype(np.float32)
    y0 = rng.uniform(0, 1, n_rows).astype(np.float32)
    return col, W, b, y0, zero


def _sweep(W, col, b, y):
    """y'[r] = sum_i W[r, i] y[col[r, i]] + b[r] (y has the zero slot last)."""
    import numpy as np

    return (W * y[col]).sum(axis=1, dtype=np.float32) + b


def _shard_worker(rank, world, port, q, iters):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2404_11894_gb300.dist import exchange_halo, shard_plan_host

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    col, W, b, y0, zero = _sweep_problem()
    L = shard_plan_host(col, zero, world, rank)
    r0, r1 = L.row_begin_own, L.row_end_own
    # local iterate: own rows, halo, zero slot
    z = np.zeros(L.local_len, np.float32)
    z[:L.rows] = y0[r0:r1]
    z[L.rows:L.rows + L.n_halo] = y0[L.halo]
    for _ in range(iters):
        send = torch.from_numpy(np.ascontiguousarray(z[L.send_idx]))
        zt = torch.from_numpy(z)
        zt[L.rows:L.rows + L.n_halo] = float("nan")  # every halo entry must arrive through the exchange
        exchange_halo(send, L, zt)
        z = zt.numpy()
        new = _sweep(W[r0:r1], L.local_col, b[r0:r1], z)
        z = z.copy()
        z[:L.rows] = new
    q.put((rank, L.row_begin.tolist(), r0, r1, z[:L.rows].copy(), L.halo.copy(), L.recv_begin.copy(),
           L.send_begin.copy(), L.send_idx.copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sweeps_equal_unsharded(world):
    """Shards of a sweep matrix on gloo ranks: the row ranges cover the rows
    with nearly equal live entries, every halo holds exactly the foreign
    columns its rows read, each rank sends a peer exactly that peer's halo
    segment, and after several sweeps with a halo exchange before each the
    shards' rows equal the unsharded sweeps bit for bit."""
    import numpy as np

    iters = 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q, iters)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=180) for _ in procs], key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    col, W, b, y0, zero = _sweep_problem()
    n = len(b)
    y = np.concatenate([y0, [0.0]]).astype(np.float32)
    for _ in range(iters):
        y = np.concatenate([_sweep(W, col, b, y), [0.0]]).astype(np.float32)
    rb = out[0][1]
    assert all(o[1] == rb for o in out) and rb[0] == 0 and rb[-1] == n
    live = (col != zero).sum(axis=1)
    per = [live[rb[p]:rb[p + 1]].sum() for p in range(world)]
    assert max(per) - min(per) <= 2 * col.shape[1]
    for rank, _, r0, r1, rows, halo, recv_begin, send_begin, send_idx in out:
        assert np.array_equal(rows, y[r0:r1])  # bitwise
        c = col[r0:r1]
        expect = np.unique(c[(c != zero) & ((c < r0) | (c >= r1))])
        assert np.array_equal(halo, expect)
        for peer in range(world):
            if peer == rank:
                continue
            # what this rank receives from peer == what peer sends to it
            seg = halo[recv_begin[peer]:recv_begin[peer + 1]]
            _, _, p0, _, _, _, _, psb, psi = out[peer]
            assert np.array_equal(seg, p0 + psi[psb[rank]:psb[rank + 1]])
            assert np.all((seg >= rb[peer]) & (seg < rb[peer + 1]))


def test_shard_plan_single_shard_has_no_halo():
    import numpy as np

    from paper_2404_11894_gb300.dist import shard_plan_host

    col, W, b, y0, zero = _sweep_problem(500)
    L = shard_plan_host(col, zero, 1, 0)
    assert L.n_halo == 0 and L.n_send == 0 and L.rows == 500
    assert np.array_equal(L.local_col, np.where(col == zero, 500, col))
