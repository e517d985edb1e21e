"""Multi-GPU story = independent replicas (rays shard with no exchange).  The
benchmark's cross-rank aggregation (max of the ranks' times, sum of their
rays) is exercised here with two gloo ranks on the CPU."""

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
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [10.0, 25.0][rank]          # rank 1 is the slow replica
    local_rays = [1000, 3000][rank]
    rate, t = bench.replica_throughput(local_ms, local_rays, steps=4, dist=dist, device="cpu")
    q.put((rank, rate, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_job_throughput_over_the_slowest_rank():
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
    for _, rate, t in got:
        assert t == pytest.approx(25.0)
        assert rate == pytest.approx((1000 + 3000) * 4 / 0.025)


def test_single_process_is_its_own_job():
    import bench
    rate, t = bench.replica_throughput(8.0, 500, steps=2)
    assert t == 8.0 and rate == pytest.approx(500 * 2 / 0.008)
