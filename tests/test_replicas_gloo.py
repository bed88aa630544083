"""The multi-process path of the benchmark on CPU: world size 2 over gloo.

The bulk path does not shard (one database per GPU, no exchange step), so N
GPUs run N independent replicas; the whole-job throughput adds the units of
every rank and divides by the slowest rank's time.  This checks that
reduction and the barrier with real processes, without a GPU.
"""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    # rank r processed 100 * (r + 1) units in (r + 1) seconds
    v = bench.replica_throughput(100.0 * (rank + 1), float(rank + 1), dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, v))


def test_replica_throughput_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # (100 + 200) units over the slowest rank's 2 seconds, seen by every rank
    assert out[0] == pytest.approx(150.0) and out[1] == pytest.approx(150.0)


def test_replica_throughput_single_process():
    import bench
    assert bench.replica_throughput(1000.0, 2.0) == 500.0
