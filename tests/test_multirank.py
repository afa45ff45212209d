"""The N-replica path of bench.py: with one process per GPU, the whole-job time is the
slowest rank's and the work is summed.  Runs as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        elapsed, total = bench.reduce_over_ranks(1.0 + rank, 10 * (rank + 1), "cpu")
        results[rank] = (elapsed, total)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    for r in range(2):
        assert results[r] == (2.0, 30.0)


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(3.5, 7, "cpu") == (3.5, 7.0)
