"""Host logic of the N > 1 bench path, on CPU with two gloo ranks: each rank times
its own replica of the window, the job's time is the slowest rank's, and the
whole-job rate counts every rank's views (the path shards only as replicas)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r took 100 * (r + 1) ms for 4 steps of a 12-view window
        ms, value = bench.whole_job_rate(100.0 * (rank + 1), 4, 12, world, torch.device("cpu"))
        dist.barrier()
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_over_ranks_and_whole_job_rate():
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
    for _, ms, value in res:
        assert ms == pytest.approx(200.0 / 4)          # the slowest rank's time
        assert value == pytest.approx(2 * 12 / 0.05)   # all ranks' views over that time


def test_single_rank_is_its_own_rate():
    import torch
    import bench
    ms, value = bench.whole_job_rate(46.54, 10, 12, 1, torch.device("cpu"))
    assert ms == pytest.approx(4.654) and value == pytest.approx(12 / 4.654e-3)
