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
