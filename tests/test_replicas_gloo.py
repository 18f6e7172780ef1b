"""The multi-GPU path of bench.py runs one replica per rank (the product has no exchange step);
the job's time is the slowest rank's and its value the products of all ranks per second. Checked
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, e2e = bench.replica_times(1.0 + rank, 5.0 - rank, dist, "cpu")
    q.put((rank, ms, e2e, bench.job_value(world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_times_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, value in out:
        assert ms == 2.0 and e2e == 5.0  # the slowest rank's step time in each measurement
        assert value == pytest.approx(1000.0)  # 2 ranks x 1 product per 2 ms


def test_single_process_is_unchanged():
    import bench
    assert bench.replica_times(3.0, 4.0, None, "cpu") == (3.0, 4.0)
    assert bench.job_value(1, 0.5) == pytest.approx(2000.0)
