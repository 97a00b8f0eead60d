"""The multi-GPU path is replicas only: every rank generates its own RVE and
the ranks exchange nothing but the timing reduction.  That reduction (max of
the times, sum of the updates over ranks) is run here with world size 2 on
the gloo backend, on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dev, e2e, upd = bench.combine_ranks(1.0 + rank, 2.0 + 3 * rank, 100.0 * (rank + 1), dist, "cpu")
        out.put((rank, dev, e2e, upd))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, dev, e2e, upd in res:
        assert dev == 2.0 and e2e == 5.0 and upd == 300.0
