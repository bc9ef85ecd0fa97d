"""Multi-GPU runs are independent replicas (the path does not shard): the only cross-rank step is
the max over ranks of the timed region and the whole-job throughput.  Checked with two gloo ranks
on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [0.25, 0.5][rank]                       # the slower replica sets the job time
    tmax = bench.replica_max(t, world, "cpu")
    value = bench.replica_throughput(1000, world, tmax)
    out.put((rank, tmax, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, value in res:
        assert tmax == 0.5
        assert value == pytest.approx(2 * 1000 / 0.5)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(0.3, 1, "cpu") == 0.3
    assert bench.replica_throughput(10, 1, 2.0) == 5.0
