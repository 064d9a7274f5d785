"""The multi-GPU form of the benchmark is independent replicas (one droplet
per rank, no data-path collective): the job's throughput is every rank's cells
x steps over the slowest rank's time.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 100.0 + 50.0 * rank          # rank 1 is the slowest: 150 ms
    value, t_max = bench.replica_throughput(t_local, 131072, 10)
    q.put((rank, value, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = 2 * 131072 * 10 / 0.150 / 1e6
    for rank, value, t_max in out:
        assert t_max == pytest.approx(150.0)
        assert value == pytest.approx(expect, rel=1e-12)


def test_replica_throughput_single_process():
    import bench
    value, t_max = bench.replica_throughput(200.0, 1000, 4)
    assert t_max == 200.0 and value == pytest.approx(1000 * 4 / 0.2 / 1e6)
