"""The multi-process path of bench.py on CPU: two gloo ranks, the k-point shard covers the path exactly once, and the
timing reduction returns the max over ranks on every rank (no collective touches the solve's data)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = bench.shard(40, rank, ws)
    got = bench.max_over_ranks(10.0 + rank, dist)
    bench.barrier(dist)
    out.put((rank, mine, got))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(40))
    assert all(r[2] == 11.0 for r in res)


@pytest.mark.parametrize("nk,ws", [(40, 3), (7, 8), (1, 2)])
def test_shard_partition(nk, ws):
    import bench
    allk = [k for r in range(ws) for k in bench.shard(nk, r, ws)]
    assert allk == list(range(nk))
