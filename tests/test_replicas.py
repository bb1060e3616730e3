"""Host-side multi-rank logic with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

from paper_2507_00254_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 1000
        off = replicas.shot_offset(rank, n)
        t = 1.5 if rank == 1 else 1.0  # rank 1 is the slow one
        tmax = replicas.max_over_ranks(t, dist)
        rate = replicas.job_rate(n, world, tmax)
        q.put((rank, off, tmax, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_ranges_and_the_slowest_time():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [0, 1000]
    assert all(r[2] == 1.5 for r in res)
    assert all(abs(r[3] - 2000 / 1.5) < 1e-9 for r in res)


def test_single_rank_helpers():
    assert replicas.max_over_ranks(2.0) == 2.0
    assert replicas.shot_offset(3, 10) == 30
    with pytest.raises(ValueError):
        replicas.job_rate(10, 1, 0.0)
