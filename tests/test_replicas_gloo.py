"""Multi-rank bookkeeping of replica runs, on CPU with the gloo backend (world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2306_07342_gb300 import replicas
    try:
        r, w, lr = replicas.env()
        replicas.barrier()
        mx = replicas.max_over_ranks(1.0 + rank)          # slowest rank decides the job time
        sm = replicas.sum_over_ranks(10.0 * (rank + 1))
        thr = replicas.job_throughput(100.0, 2.0 + rank)   # 200 units over the slowest 3.0 s
        mine = replicas.shard(list(range(7)), r, w)
        q.put((rank, r, w, lr, mx, sm, thr, mine))
    finally:
        dist.destroy_process_group()


def test_replica_bookkeeping_world_size_2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    shards = []
    for rank, r, w, lr, mx, sm, thr, mine in res:
        assert (r, w, lr) == (rank, 2, rank)
        assert mx == 2.0 and sm == 30.0
        assert abs(thr - 200.0 / 3.0) < 1e-12
        shards += mine
    assert sorted(shards) == list(range(7))


def test_single_process_defaults():
    from paper_2306_07342_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10.0, 2.0) == 5.0
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
