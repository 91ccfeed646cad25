"""Multi-GPU runs of the benchmark are independent replicas (the sort of one
array does not shard here): every rank sorts its own array and the job's
throughput is all ranks' keys over the slowest rank's time.  The aggregation
runs as world_size-2 gloo ranks on CPU."""
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
    total_ms = [30.0, 50.0][rank]                       # rank 1 is the slowest
    ms, value = bench.aggregate_over_ranks(total_ms, keys_per_rank=10**6, steps=10, world=world)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == pytest.approx(5.0)                 # 50 ms over 10 steps, the max
        assert value == pytest.approx(2 * 10**6 / 5e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_over_ranks(40.0, keys_per_rank=10**8, steps=10, world=1)
    assert ms == pytest.approx(4.0) and value == pytest.approx(25.0)
